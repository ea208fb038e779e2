// C ABI of the GB300 phMG library (include/stokes_mg.h): device data of the
// hierarchy, setup (patch gather, batched Gauss-Jordan, coarse bordered
// inverse, Arnoldi lambda_max), the V-cycle (Eq. 3.1 / 3.2 with Chebyshev-
// wrapped additive Schwarz, Eq. 3.4), FGMRES (Sec. 4) and the per-step
// entry points used by the parity tests.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <memory>
#include <atomic>
#include <condition_variable>
#include <exception>
#include <mutex>
#include <thread>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/stokes_mg.h"
#include "fem.hpp"
#include "assembly.cuh"
#include "kernels.cuh"
#include "batched.cuh"

namespace {

thread_local std::string g_last_error;

struct StokesError : std::runtime_error {
    int code;
    StokesError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            throw StokesError(e_ == cudaErrorMemoryAllocation ? STOKES_EOOM : STOKES_ECUDA,        \
                              std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

double host_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// STOKES_TRACE=1 prints the host timeline of setup to stderr.
bool trace_on() {
    static const bool on = [] {
        const char* e = std::getenv("STOKES_TRACE");
        return e && e[0] == '1';
    }();
    return on;
}
void trace(const char* what, int level, double t0) {
    if (trace_on()) std::fprintf(stderr, "[stokes] %-28s level %d  %8.3f ms\n", what, level, host_ms() - t0);
}

template <typename T>
T* dalloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    CK(cudaMalloc(&p, n * sizeof(T)));
    return (T*)p;
}

// One host thread that issues the device side of setup (uploads, kernel
// launches) in submission order, so that it overlaps with the assembly of
// the next level on the calling thread.  The first exception is kept and
// rethrown by finish(); later tasks are skipped.
class Launcher {
  public:
    Launcher() : th_([this] { loop(); }) {}
    ~Launcher() {
        if (th_.joinable()) {
            {
                std::lock_guard<std::mutex> g(mu_);
                stop_ = true;
            }
            cv_.notify_all();
            th_.join();
        }
    }
    void submit(std::function<void()> f) {
        {
            std::lock_guard<std::mutex> g(mu_);
            q_.push_back(std::move(f));
        }
        cv_.notify_all();
    }
    void finish() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        th_.join();
        if (err_) std::rethrow_exception(err_);
    }

  private:
    void loop() {
        for (;;) {
            std::function<void()> f;
            {
                std::unique_lock<std::mutex> lk(mu_);
                cv_.wait(lk, [&] { return stop_ || !q_.empty(); });
                if (q_.empty()) return;
                f = std::move(q_.front());
                q_.erase(q_.begin());
            }
            if (err_) continue;
            try {
                f();
            } catch (...) {
                err_ = std::current_exception();
            }
        }
    }
    std::mutex mu_;
    std::condition_variable cv_;
    std::vector<std::function<void()>> q_;
    bool stop_ = false;
    std::exception_ptr err_;
    std::thread th_;
};



inline int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}

struct DevCSR {
    int nr = 0, nc = 0;
    long long nnz = 0;
    int lanes = 16;
    int *rp = nullptr, *ci = nullptr;
    double* v64 = nullptr;
    float* v32 = nullptr;
};

struct DevLevel {
    int n = 0;
    bool p_level = false;
    DevCSR K, P, R;
    // patches
    int npatch = 0, maxn = 0;
    long long nent = 0, nsq = 0;
    int *poff = nullptr, *pdofs = nullptr, *pnv = nullptr;
    long long *moff = nullptr, *ioff64 = nullptr, *ioff32 = nullptr;
    long long saddle_smem = 0;      // max scratch (doubles) of the patches inverted in shared memory
    long long saddle_smem_fac = 0;  // the same for the factored-only inversion
    long long saddle_global = 0;    // total scratch (doubles) of the others
    long long* scoff = nullptr;     // their offsets into the global scratch
    long long ninv64 = 0, ninv32 = 0;
    double* inv64 = nullptr;            // explicit inverses (Gauss-Jordan patches; FP32 also for the batched path)
    float* inv32 = nullptr;
    // factored saddle inverses (Li, W, Si per patch; saddle_core), the stored
    // form of the saddle-block solver: FP64 on FP64 handles, FP32 on MIXED
    bool factored = false;
    long long *foff64 = nullptr, *foff32 = nullptr;
    long long nfac64 = 0, nfac32 = 0;
    double* fac64 = nullptr;
    float* fac32 = nullptr;
    int sa_xs = 0;                      // saddle apply: largest patch
    long long sa_ws64 = 0, sa_ws32 = 0; // saddle apply: largest W (elements)
    int sa_buf = 0;                     // bulk-copy apply: buffer bytes (0: not used on this level)
    bool fac_packed = false;            // L^-1 stored as its packed upper triangle (bulk-copy apply only)
    double* wt64 = nullptr;
    float* wt32 = nullptr;
    int *soff = nullptr, *sidx = nullptr;
    double* Y64 = nullptr;
    float* Y32 = nullptr;
    // V-cycle work vectors (both precisions)
    double *b64 = nullptr, *e64 = nullptr, *r64 = nullptr, *d64 = nullptr, *t64 = nullptr, *u64 = nullptr;
    float *b32 = nullptr, *e32 = nullptr, *r32 = nullptr, *d32 = nullptr, *t32 = nullptr, *u32 = nullptr;
    double lmax = 0;
    // device assembly of K (all levels but the coarsest)
    bool dev_asm = false;
    bool dev_transfer = false;          // P, R built on the device (exact nnz read back at finish)
    bool maps_up = false;               // the DoF maps the device transfers read are uploaded
    sasm::AsmMesh am;
    double* cellgeo = nullptr;          // am.cg, filled on the device
    int* asm_len = nullptr;
    int* asm_tmp = nullptr;
    int* asm_status = nullptr;
};

// Scratch of one Arnoldi run (one per relaxed level, so that levels can
// run concurrently on their own streams)
struct KrylovWS {
    double *V = nullptr, *h = nullptr, *y = nullptr, *hn = nullptr, *partial = nullptr, *v0 = nullptr;
    unsigned int* ticket = nullptr;
};

struct PendingPatches {
    int level = 0;
    double* work = nullptr;
    int* status = nullptr;
    cudaStream_t stream = nullptr;
};

struct Prof {
    bool on = false;
    long long launches = 0;
    double total_ms = 0;
    std::vector<double> each_ms;        // resolved launches, in launch order
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

// FBF(phMG) mode (Eq. fbf): the handle's levels are the scalar velocity
// hierarchy of A~^-1; the outer FGMRES works on the SV Stokes system of the
// finest level, kept here with the pressure mass blocks of S~^-1.
struct FbfData {
    sfem::Level S0;                    // the finest SV level (host-assembled K, Mv, KfD, spaces)
    int nS = 0, nu = 0, nvf = 0;       // Stokes free DoFs, free velocity DoFs, per component
    int ncell = 0, nbq = 0;            // finest cells, pressure nodes per cell
    DevLevel S0d;                      // its device assembly: K (FP64) and the inputs of the matrix-free load
    double *a = nullptr, *t = nullptr, *w = nullptr, *r = nullptr;
    double* minv = nullptr;            // [nbq][nbq] inverse reference pressure mass matrix
    double* scale = nullptr;           // [ncell] -nu_e / |det J_e|
    int* qcell = nullptr;              // [ncell][nbq] pressure nodes of each cell
};

}  // namespace

struct stokes_mg {
    int device = 0;
    stokes_mg_opts opts;
    sfem::Hierarchy H;
    std::vector<DevLevel> L;
    int dim = 2, family = 0, k = 2;
    // coarse bordered inverse
    int nc = 0;
    double* Cinv = nullptr;
    // FGMRES
    int restart = 30;
    double *V = nullptr, *Z = nullptr, *Hh = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *h = nullptr, *hn = nullptr, *resid = nullptr, *partial = nullptr, *scal = nullptr;
    double* pinned = nullptr;
    int* pinned_rb = nullptr;            // setup readback: statuses and sizes (finish_setup)
    size_t n_rb = 0;
    double* pinned_H = nullptr;          // [STOKES_MAX_LEVELS + 1][HESS_MAX * HESS_MAX]
    double* Hlev = nullptr;              // device Hessenberg matrices, one per level
    double* v0buf = nullptr;             // Arnoldi start vector
    int arn_m[STOKES_MAX_LEVELS] = {0};
    int partial_blocks = 0;
    unsigned int* ticket = nullptr;
    // V-cycle graph I/O
    double *vin = nullptr, *vout = nullptr;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    long long graph_launches[2] = {0, 0};
    // batched V-cycle: interleaved work vectors of width bm per level, and
    // one captured graph per patch-GEMM mode for that width
    // one launch of the batched patch GEMM: `count` patches of one kind from
    // the level's size-sorted patch list, starting at `off` (sizes lo .. hi)
    struct GemmPart { int kind = 0, nw = 0, off = 0, count = 0, lo = 0, hi = 0; double us = 0; };
    struct BatchLevel {
        float *b = nullptr, *e = nullptr, *r = nullptr, *d = nullptr, *t = nullptr, *u = nullptr, *Yb = nullptr;
        std::vector<GemmPart> plan[2];   // per mode, empty until the first batched use at this width
        double single_us[2] = {0, 0};    // the level as one launch per kind (the untuned plan), timed alongside
    };
    std::vector<int*> bpsort;            // per relaxed level: patch indices sorted by size (device)
    int bm = 0;
    std::vector<BatchLevel> bl;
    int *bstat_h = nullptr, *bstat_d = nullptr;   // host-mapped timeout flag of the tensor-core patch GEMM
    std::vector<void*> tmaps;                      // per relaxed level: tensor maps over the FP32 inverses
    std::vector<void*> tmaps_hi, tmaps_lo;         // per relaxed level: over their TF32 hi / lo parts (3xTF32)
    std::vector<float*> inv_hi, inv_lo;            // per relaxed level: the hi / lo parts
    std::unique_ptr<FbfData> fbf;                  // FBF(phMG) mode (stokes_fbf_setup)
    // batched FGMRES workspace (interleaved FP64, width bk_m)
    struct BatchKrylov {
        int m = 0;
        double *V = nullptr, *Z = nullptr, *W = nullptr, *R = nullptr, *B = nullptr, *X = nullptr, *partial = nullptr;
        double *hcol = nullptr, *hcol2 = nullptr, *hn = nullptr, *Hc = nullptr, *cs = nullptr, *sn = nullptr;
        double *g = nullptr, *y = nullptr, *resid = nullptr, *beta = nullptr, *beta0 = nullptr;
        double* host = nullptr;        // pinned [2 m]
        int io_m = 0;                  // width of the batched solve's free-DoF buffers
        double *iob = nullptr, *iox = nullptr;
    } bk;
    cudaGraphExec_t bgraph[2] = {nullptr, nullptr};
    long long bgraph_launches[2] = {0, 0};
    // solve plumbing (finest level)
    DevCSR Mv, KfD;
    int *vel_rows = nullptr;    // free velocity row -> full velocity index
    double *F = nullptr, *bvec = nullptr, *xvec = nullptr, *ones = nullptr, *pint = nullptr, *gzero = nullptr;
    double pint_sum = 0;
    // stats / profiling
    stokes_mg_stats st;
    long long launches = 0;
    Prof prof[5];
    bool capturing = false;
    bool host_only = false;
    int* sa_status = nullptr;           // device: 1 once a bulk-copy apply CTA gave up waiting
    // programmatic dependent launch inside a V-cycle's chain of kernels:
    // pdl_chain while the chain is issued, pdl_armed once a kernel of the
    // chain precedes the next launch on the stream (a copy disarms it)
    bool pdl_chain = false;
    bool pdl_armed = false;
    // bump allocator for the handle's long-lived device buffers: a few large
    // cudaMalloc chunks instead of one call per array
    char* slab_cur = nullptr;
    size_t slab_left = 0;
    std::vector<void*> pool_allocs;      // freed to the device pool at destroy
    // setup in flight
    std::vector<PendingPatches> pending;
    int* c_ipiv = nullptr;
    double* c_colk = nullptr;
    int* c_status = nullptr;
    cudaStream_t s_up = nullptr, s_coarse = nullptr;
    std::vector<KrylovWS> kws;           // per relaxed level (level 0 aliases the FGMRES buffers)
    std::vector<cudaStream_t> s_lvl;     // setup compute stream of each relaxed level
    std::vector<double*> mesh_X;         // device vertex coordinates per mesh
    std::vector<int*> mesh_C;            // device cells per mesh
    std::vector<int*> mesh_parent;       // device parent map per mesh (cell -> next coarser mesh's cell)
    cudaStream_t s_tr = nullptr;         // setup stream of the device transfers
    std::vector<void*> allocs;
    // STOKES_TRACE=1: device timeline of setup (event, label, host time)
    struct Mark { std::string what; double host, dev; };
    std::vector<Mark*> marks;
    std::mutex marks_mu;
};

namespace {

enum ProfKind { PK_PATCH = 0, PK_SPMV = 1, PK_GJ = 2, PK_PULL = 3, PK_TRANSFER = 4 };

// the Stokes level the solve works on: the finest level of the hierarchy, or
// in FBF mode the SV level kept beside the scalar velocity hierarchy
const sfem::Level& finest_stokes(const stokes_mg* h) { return h->fbf ? h->fbf->S0 : h->H.levels[0]; }

template <typename F>
void launch(stokes_mg* h, int kind, cudaStream_t s, F&& f) {
    Prof* p = (kind >= 0 && kind < 5) ? &h->prof[kind] : nullptr;
    bool ev = p && p->on && !h->capturing;
    cudaEvent_t a = nullptr, b = nullptr;
    if (ev) {
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(a, s));
    }
    f();
    CK(cudaGetLastError());
    h->launches++;
    if (ev) {
        CK(cudaEventRecord(b, s));
        p->pending.push_back({a, b});
        p->launches++;
    }
}

// One kernel launch.  While a V-cycle chain is issued (pdl_chain) every
// kernel after the chain's first is launched with programmatic stream
// serialisation: its blocks may be scheduled while the kernel before it
// finishes, and wait (skern::pdl_wait) before they touch what that kernel
// writes.  Only kernels that call pdl_wait go through here.
template <typename... KArgs, typename... Args>
void kl(stokes_mg* h, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    if (h->pdl_armed) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CK(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
    } else {
        kern<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
    }
    h->pdl_armed = h->pdl_chain;
}

// Device timeline of setup under STOKES_TRACE=1: a host function enqueued
// on `s` stamps the time at which the stream reaches this point; print_marks
// lists the stamps against the first one.
void mark_cb(void* p) { static_cast<stokes_mg::Mark*>(p)->dev = host_ms(); }
void mark(stokes_mg* h, const std::string& what, cudaStream_t s) {
    if (!trace_on()) return;
    stokes_mg::Mark* m = new stokes_mg::Mark{what, host_ms(), 0.0};
    {
        std::lock_guard<std::mutex> g(h->marks_mu);
        h->marks.push_back(m);
    }
    CK(cudaLaunchHostFunc(s, mark_cb, m));
}
void print_marks(stokes_mg* h) {
    if (h->marks.empty()) return;
    CK(cudaDeviceSynchronize());
    const double t0 = h->marks[0]->host;
    for (auto* m : h->marks) {
        std::fprintf(stderr, "[stokes] %-34s device %8.3f ms  issued %8.3f ms\n", m->what.c_str(), m->dev - t0,
                     m->host - t0);
        delete m;
    }
    h->marks.clear();
}

template <typename T>
T* track(stokes_mg* h, T* p) {
    h->allocs.push_back((void*)p);
    return p;
}

// Process-wide stream-ordered memory pool per device.  Its release
// threshold is unlimited, so memory freed by one handle stays reserved and
// the next setup allocates without touching the driver's allocator (a plain
// cudaMalloc issued while the patch inversion runs was observed to wait for it).
cudaMemPool_t device_pool(int dev) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {nullptr};
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) throw StokesError(STOKES_EUNSUPPORTED, "device index beyond 64");
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CK(cudaMemPoolCreate(&pools[dev], &props));
        unsigned long long thr = ~0ULL;
        CK(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &thr));
    }
    return pools[dev];
}

template <typename T>
T* palloc(int dev, size_t n, cudaStream_t s) {
    void* p = nullptr;
    if (n == 0) n = 1;
    CK(cudaMallocFromPoolAsync(&p, n * sizeof(T), device_pool(dev), s));
    return (T*)p;
}

constexpr size_t kSlabChunk = size_t(256) << 20;

// Device buffer owned by the handle (freed by stokes_mg_destroy), 256-byte
// aligned, carved from 256 MB chunks; large requests get their own chunk.
template <typename T>
T* halloc(stokes_mg* h, size_t n) {
    size_t bytes = ((std::max<size_t>(n, 1) * sizeof(T)) + 255) & ~size_t(255);
    if (bytes > kSlabChunk / 4) {
        T* p = palloc<T>(h->device, n, h->s_up);
        h->pool_allocs.push_back((void*)p);
        return p;
    }
    if (h->slab_left < bytes) {
        h->slab_cur = palloc<char>(h->device, kSlabChunk, h->s_up);
        h->pool_allocs.push_back((void*)h->slab_cur);
        h->slab_left = kSlabChunk;
    }
    T* p = (T*)h->slab_cur;
    h->slab_cur += bytes;
    h->slab_left -= bytes;
    return p;
}

// Host-to-device upload into the handle's memory.  On Grace-based GB300
// nodes pageable copies run over NVLink-C2C through the host page tables
// (measured ~165 GB/s, against ~13 GB/s for a single-threaded host copy into
// a pinned staging buffer), so arrays are copied straight from their
// pageable host vectors.
template <typename Vec>
typename Vec::value_type* hupload(stokes_mg* h, const Vec& v, cudaStream_t s) {
    using T = typename Vec::value_type;
    T* p = halloc<T>(h, v.size());
    const size_t bytes = v.size() * sizeof(T);
    if (bytes) CK(cudaMemcpyAsync(p, v.data(), bytes, cudaMemcpyHostToDevice, s));
    return p;
}

// Lanes per row of the CSR SpMV: with four entries per lane per round, four
// lanes cover a row of up to ~64 entries in a few rounds with fewer idle
// lanes and shuffle steps than wider groups (measured fastest for the
// Stokes operators, FP32 and FP64, whose rows hold ~25-120 entries).
int choose_lanes(const DevCSR& A) {
    double avg = A.nr ? (double)A.nnz / A.nr : 1;
    if (avg <= 64) return 4;
    if (avg <= 128) return 8;
    return 16;
}

DevCSR upload_csr(stokes_mg* h, const sfem::CSR& A, bool want32, cudaStream_t s) {
    DevCSR d;
    d.nr = A.nr;
    d.nc = A.ncol;
    d.nnz = A.nnz();
    d.rp = hupload(h, A.rp, s);
    d.ci = hupload(h, A.ci, s);
    d.v64 = hupload(h, A.v, s);
    if (want32) {
        d.v32 = halloc<float>(h, d.nnz);
        skern::convert_vec<float, double><<<grid_for(d.nnz), 256, 0, s>>>((int)d.nnz, d.v64, d.v32);
        CK(cudaGetLastError());
    }
    d.lanes = choose_lanes(d);
    return d;
}

template <typename T>
const T* vals(const DevCSR& A);
template <>
const double* vals<double>(const DevCSR& A) { return A.v64; }
template <>
const float* vals<float>(const DevCSR& A) { return A.v32; }

// lanes per row for an FP32 operator: 8 for rows of 33-64 entries (measured
// 8-13% faster than 4 on the 64x64 P4 operator, 41 entries per row); an FP64
// operator keeps the 4 of choose_lanes there
int lanes_for(const DevCSR& A, size_t elem) {
    const double avg = A.nr ? (double)A.nnz / A.nr : 1;
    return elem == 4 && avg > 32 && avg <= 64 ? 8 : A.lanes;
}

template <typename T, int MODE>
void spmv_lanes(stokes_mg* h, const DevCSR& A, const T* x, T* y, const T* b, cudaStream_t s) {
    const int lanes = lanes_for(A, sizeof(T));
    const long long threads = (long long)A.nr * lanes;
    const int grid = (int)((threads + 255) / 256);
    if (A.nr == 0) return;
    const T* av = vals<T>(A);
    switch (lanes) {
        case 4: kl(h, skern::spmv_csr<T, 4, MODE>, grid, 256, 0, s, A.nr, A.rp, A.ci, av, x, y, b); break;
        case 8: kl(h, skern::spmv_csr<T, 8, MODE>, grid, 256, 0, s, A.nr, A.rp, A.ci, av, x, y, b); break;
        case 16: kl(h, skern::spmv_csr<T, 16, MODE>, grid, 256, 0, s, A.nr, A.rp, A.ci, av, x, y, b); break;
        default: kl(h, skern::spmv_csr<T, 32, MODE>, grid, 256, 0, s, A.nr, A.rp, A.ci, av, x, y, b); break;
    }
}

template <typename T>
void spmv(stokes_mg* h, int kind, const DevCSR& A, int mode, const T* x, T* y, const T* b, cudaStream_t s) {
    launch(h, kind, s, [&] {
        if (mode == skern::SPMV_SET) spmv_lanes<T, skern::SPMV_SET>(h, A, x, y, b, s);
        else if (mode == skern::SPMV_ADD) spmv_lanes<T, skern::SPMV_ADD>(h, A, x, y, b, s);
        else spmv_lanes<T, skern::SPMV_RESID>(h, A, x, y, b, s);
    });
}

// ---- per-precision accessors of a level
template <typename T> struct LV;
template <> struct LV<double> {
    static double* b(DevLevel& l) { return l.b64; }
    static double* e(DevLevel& l) { return l.e64; }
    static double* r(DevLevel& l) { return l.r64; }
    static double* d(DevLevel& l) { return l.d64; }
    static double* t(DevLevel& l) { return l.t64; }
    static double* u(DevLevel& l) { return l.u64; }
};
template <> struct LV<float> {
    static float* b(DevLevel& l) { return l.b32; }
    static float* e(DevLevel& l) { return l.e32; }
    static float* r(DevLevel& l) { return l.r32; }
    static float* d(DevLevel& l) { return l.d32; }
    static float* t(DevLevel& l) { return l.t32; }
    static float* u(DevLevel& l) { return l.u32; }
};

// The bulk-copy apply's bounded waits report through h->sa_status: read it
// (one int, after the stream's work) and fail with ECUDA if a CTA gave up.
void check_sa_status(stokes_mg* h, cudaStream_t s) {
    if (!h->sa_status) return;
    int v = 0;
    CK(cudaMemcpyAsync(&v, h->sa_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (v != 0)
        throw StokesError(STOKES_ECUDA, "a patch-apply CTA gave up waiting for its bulk copy (bounded wait)");
}

// per-precision patch data and apply kernels of a level
template <typename T> struct PatchOf;
template <> struct PatchOf<float> {
    static const float* fac(const DevLevel& l) { return l.fac32; }
    static const long long* foff(const DevLevel& l) { return l.foff32; }
    static const float* inv(const DevLevel& l) { return l.inv32; }
    static const long long* ioff(const DevLevel& l) { return l.ioff32; }
    static const float* wt(const DevLevel& l) { return l.wt32; }
    static float* Y(const DevLevel& l) { return l.Y32; }
    static long long ws(const DevLevel& l) { return l.sa_ws32; }
    static constexpr auto bulk = skern::saddle_apply_bulk_f32;
    static constexpr auto fact = skern::saddle_apply_f32;
    static constexpr auto expl = skern::patch_apply_f32;
    static constexpr int vec = 4;
    static constexpr size_t red = sizeof(float4);
    static constexpr const char* none = "no FP32 patch inverses on this handle (FP64 handle)";
};
template <> struct PatchOf<double> {
    static const double* fac(const DevLevel& l) { return l.fac64; }
    static const long long* foff(const DevLevel& l) { return l.foff64; }
    static const double* inv(const DevLevel& l) { return l.inv64; }
    static const long long* ioff(const DevLevel& l) { return l.ioff64; }
    static const double* wt(const DevLevel& l) { return l.wt64; }
    static double* Y(const DevLevel& l) { return l.Y64; }
    static long long ws(const DevLevel& l) { return l.sa_ws64; }
    static constexpr auto bulk = skern::saddle_apply_bulk_f64;
    static constexpr auto fact = skern::saddle_apply_f64;
    static constexpr auto expl = skern::patch_apply_f64;
    static constexpr int vec = 2;
    static constexpr size_t red = sizeof(double2);
    static constexpr const char* none = "no FP64 patch inverses on this handle (MIXED handle)";
};

// one ASM sweep: Y = W_i K_i^{-1} I_i r for every patch, then
// out = alpha * sum_i I_i^T Y_i + beta * out in the same pass as the
// Chebyshev bookkeeping: x = out or x += out (xmode), rdst = bsrc (if rdst)
template <typename T>
void asm_apply(stokes_mg* h, DevLevel& l, const T* r, T* out, double alpha, double beta, cudaStream_t s,
               T* x = nullptr, int xmode = skern::PULL_X_NONE, const T* bsrc = nullptr, T* rdst = nullptr) {
    using PO = PatchOf<T>;
    const T* fac = PO::fac(l);
    const long long* foff = PO::foff(l);
    const T* wt = PO::wt(l);
    T* Y = PO::Y(l);
    const int *poff = l.poff, *pdofs = l.pdofs, *pnv = l.pnv;
    if (fac && l.sa_buf > 0) {
        const size_t smem = skern::saddle_apply_bulk_smem(l.sa_buf, sizeof(T), l.sa_xs);
        launch(h, PK_PATCH, s, [&] {
            kl(h, PO::bulk, l.npatch, skern::SA_BULK_THREADS, smem, s, h->dim, poff, pdofs, pnv, foff, fac, r, wt, Y,
               (int)l.sa_buf, (int)l.sa_xs, h->sa_status);
        });
    } else if (fac) {
        long long ws = PO::ws(l);
        if (skern::saddle_apply_smem(sizeof(T), PO::vec, ws, l.sa_xs) > skern::SADDLE_APPLY_SMEM_MAX) ws = 0;
        const size_t smem = skern::saddle_apply_smem(sizeof(T), PO::vec, ws, l.sa_xs);
        launch(h, PK_PATCH, s, [&] {
            kl(h, PO::fact, l.npatch, skern::SADDLE_APPLY_THREADS, smem, s, l.npatch, h->dim, poff, pdofs, pnv, foff,
               fac, r, wt, Y, (int)l.sa_xs, (int)ws);
        });
    } else {
        const T* inv = PO::inv(l);
        if (!inv) throw StokesError(STOKES_EINVAL, PO::none);
        const size_t smem = PO::red * (128 + 4) + sizeof(T) * l.maxn;
        launch(h, PK_PATCH, s, [&] {
            kl(h, PO::expl, l.npatch, 128, smem, s, l.npatch, poff, pdofs, PO::ioff(l), inv, r, wt, Y);
        });
    }
    const int *soff = l.soff, *sidx = l.sidx;
    launch(h, PK_PULL, s, [&] {
        kl(h, skern::pull_scatter<T>, grid_for(l.n), 256, 0, s, l.n, soff, sidx, (const T*)Y, (T)alpha, (T)beta, out, x,
           xmode, bsrc, rdst);
    });
}

template <typename T>
void axpby_l(stokes_mg* h, int n, double a, const T* x, double b, T* y, cudaStream_t s) {
    launch(h, -1, s, [&] { kl(h, skern::axpby<T>, grid_for(n), 256, 0, s, n, (T)a, x, (T)b, y); });
}

// Chebyshev(nu) preconditioned by one ASM sweep per step, on [lo, hi]*lmax
// (three-term recurrence); x_zero: x starts at 0.
template <typename T>
void smooth(stokes_mg* h, int li, const T* b, T* x, bool x_zero, int nu, cudaStream_t s) {
    DevLevel& l = h->L[li];
    const double a = h->opts.cheb_lo * l.lmax, bb = h->opts.cheb_hi * l.lmax;
    const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
    double rho = 1.0 / sigma;
    T* r = LV<T>::r(l);
    const T* rin;
    if (x_zero) {
        rin = b;
    } else {
        spmv<T>(h, PK_SPMV, l.K, skern::SPMV_RESID, x, r, b, s);
        rin = r;
    }
    if (nu == 1) {
        asm_apply<T>(h, l, rin, x, 1.0 / theta, x_zero ? 0.0 : 1.0, s);
        return;
    }
    // d = M r (step 1), then x = d and r = b from x = 0, else x += d; every
    // later step: r -= K d, d = (2 rho_i / delta) M r + rho_i rho_{i-1} d,
    // x += d (the updates of x and the copy of b ride in the scatter pass)
    T* d = LV<T>::d(l);
    if (x_zero) asm_apply<T>(h, l, rin, d, 1.0 / theta, 0.0, s, x, skern::PULL_X_SET, b, r);
    else asm_apply<T>(h, l, rin, d, 1.0 / theta, 0.0, s, x, skern::PULL_X_ADD);
    for (int i = 1; i < nu; ++i) {
        spmv<T>(h, PK_SPMV, l.K, skern::SPMV_RESID, d, r, r, s);    // r -= K d
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        asm_apply<T>(h, l, r, d, 2.0 * rho_new / delta, rho_new * rho, s, x, skern::PULL_X_ADD);
        rho = rho_new;
    }
}

// e = C^-1 (b, 0) on the bordered coarse inverse, in FP64 (an FP32 b is
// widened exactly and e rounded once, in the same kernel)
template <typename T>
void coarse_apply(stokes_mg* h, const T* b, T* e, cudaStream_t s) {
    const int n = h->nc;
    launch(h, -1, s, [&] {
        kl(h, skern::dense_gemv<T, T>, (n * 32 + 255) / 256, 256, 0, s, n, n, n + 1, (const double*)h->Cinv, b, e);
    });
}

// hMG V-cycle (Eq. 3.1, Fig. 2) on level li from e = 0
template <typename T>
void hcycle(stokes_mg* h, int li, const T* b, T* e, cudaStream_t s) {
    const int last = (int)h->L.size() - 1;
    if (li == last) { coarse_apply<T>(h, b, e, s); return; }
    DevLevel& l = h->L[li];
    DevLevel& c = h->L[li + 1];
    const int nu = h->opts.nu_h;
    smooth<T>(h, li, b, e, true, nu, s);
    spmv<T>(h, PK_SPMV, l.K, skern::SPMV_RESID, e, LV<T>::r(l), b, s);
    spmv<T>(h, PK_TRANSFER, l.R, skern::SPMV_SET, LV<T>::r(l), LV<T>::b(c), (const T*)nullptr, s);
    hcycle<T>(h, li + 1, LV<T>::b(c), LV<T>::e(c), s);
    spmv<T>(h, PK_TRANSFER, l.P, skern::SPMV_ADD, LV<T>::e(c), e, (const T*)nullptr, s);
    smooth<T>(h, li, b, e, false, nu, s);
}

// phMG cycle: defect correction (Eq. 3.2) on the p-levels; the first hMG
// level runs n_V hMG cycles, each on the current defect.
template <typename T>
void pcycle(stokes_mg* h, int li, const T* b, T* e, cudaStream_t s) {
    const int last = (int)h->L.size() - 1;
    if (li == last) { coarse_apply<T>(h, b, e, s); return; }
    DevLevel& l = h->L[li];
    if (!l.p_level) {
        hcycle<T>(h, li, b, e, s);
        for (int t = 1; t < h->opts.n_V; ++t) {
            spmv<T>(h, PK_SPMV, l.K, skern::SPMV_RESID, e, LV<T>::t(l), b, s);
            hcycle<T>(h, li, LV<T>::t(l), LV<T>::u(l), s);
            axpby_l<T>(h, l.n, 1.0, LV<T>::u(l), 1.0, e, s);
        }
        return;
    }
    DevLevel& c = h->L[li + 1];
    const int nu = h->opts.nu_p;
    smooth<T>(h, li, b, e, true, nu, s);
    spmv<T>(h, PK_SPMV, l.K, skern::SPMV_RESID, e, LV<T>::r(l), b, s);
    spmv<T>(h, PK_TRANSFER, l.R, skern::SPMV_SET, LV<T>::r(l), LV<T>::b(c), (const T*)nullptr, s);
    pcycle<T>(h, li + 1, LV<T>::b(c), LV<T>::e(c), s);
    spmv<T>(h, PK_TRANSFER, l.P, skern::SPMV_ADD, LV<T>::e(c), e, (const T*)nullptr, s);
    smooth<T>(h, li, b, e, false, nu, s);
}

// vout = B_MG vin in the requested precision (vin/vout are the FP64 graph
// I/O buffers).  With pdl, every kernel after the first is launched with
// programmatic dependent launch (the body issues kernels only).
void vcycle_body(stokes_mg* h, int prec, cudaStream_t s, bool pdl = true) {
    DevLevel& l0 = h->L[0];
    const int n = l0.n;
    h->pdl_chain = pdl;
    h->pdl_armed = false;
    try {
        if (prec == STOKES_FP64) {
            pcycle<double>(h, 0, h->vin, h->vout, s);
        } else {
            launch(h, -1, s, [&] { kl(h, skern::convert_vec<float, double>, grid_for(n), 256, 0, s, n, (const double*)h->vin, l0.b32); });
            pcycle<float>(h, 0, l0.b32, l0.e32, s);
            launch(h, -1, s, [&] { kl(h, skern::convert_vec<double, float>, grid_for(n), 256, 0, s, n, (const float*)l0.e32, h->vout); });
        }
    } catch (...) {
        h->pdl_chain = h->pdl_armed = false;
        throw;
    }
    h->pdl_chain = h->pdl_armed = false;
}

void vcycle_run(stokes_mg* h, int prec, cudaStream_t s) {
    // per-launch events cannot sit inside a replayed graph: profiling any
    // V-cycle kernel class runs the V-cycle as plain launches
    const bool any_prof = h->prof[PK_PATCH].on || h->prof[PK_SPMV].on || h->prof[PK_PULL].on || h->prof[PK_TRANSFER].on;
    if (h->graph[prec] && !any_prof) {
        CK(cudaGraphLaunch(h->graph[prec], s));
        h->launches += h->graph_launches[prec];
    } else {
        vcycle_body(h, prec, s, !any_prof);
    }
}

void capture_graph(stokes_mg* h, int prec, cudaStream_t s) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    long long before = h->launches;
    h->capturing = true;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        vcycle_body(h, prec, cs);
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cs, &dummy);
        h->capturing = false;
        cudaStreamDestroy(cs);
        throw;
    }
    CK(cudaStreamEndCapture(cs, &g));
    h->capturing = false;
    h->graph_launches[prec] = h->launches - before;
    h->launches = before;
    CK(cudaGraphInstantiate(&h->graph[prec], g, 0));
    CK(cudaGraphDestroy(g));
    CK(cudaStreamDestroy(cs));
    (void)s;
}

// ---- batched V-cycle (m interleaved right-hand sides, FP32 operators) -----
// The same cycle as pcycle / hcycle / smooth (Eq. 3.2 / 3.1, Chebyshev around
// one ASM sweep), with SpMM for the SpMVs and transfers, the patch apply as a
// per-patch GEMM on the tensor cores (sbat::patch_gemm, mode gm) and the
// dense FP64 coarse inverse applied to the whole batch.
using BatchLevel = stokes_mg::BatchLevel;

void b_spmm(stokes_mg* h, int kind, const DevCSR& A, int mode, int m, const float* X, float* Y, const float* B,
            cudaStream_t s) {
    launch(h, kind, s, [&] { sbat::spmm(mode, A.nr, m, A.rp, A.ci, A.v32, X, Y, B, s); });
}

const void* split_map(const std::vector<void*>& v, size_t li) { return li < v.size() ? v[li] : nullptr; }

void b_asm(stokes_mg* h, int li, int gm, int m, const float* r, float* out, double alpha, double beta, cudaStream_t s) {
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    if (B.plan[gm].empty()) throw StokesError(STOKES_ECUDA, "internal: no batched patch GEMM plan for this level");
    for (const auto& pt : B.plan[gm])
        launch(h, PK_PATCH, s, [&] {
            sbat::patch_gemm(gm, pt.kind, pt.nw, pt.count, h->bpsort[li] + pt.off, pt.hi, m, l.poff, l.pdofs, l.ioff32,
                             l.inv32, h->tmaps[li], split_map(h->tmaps_hi, li), split_map(h->tmaps_lo, li), r, l.wt32,
                             B.Yb, h->bstat_d, s);
        });
    launch(h, PK_PULL, s, [&] { sbat::pull_scatter(l.n, m, l.soff, l.sidx, B.Yb, (float)alpha, (float)beta, out, s); });
}

void b_smooth(stokes_mg* h, int li, int gm, int m, const float* b, float* x, bool x_zero, int nu, cudaStream_t s) {
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    const double a = h->opts.cheb_lo * l.lmax, bb = h->opts.cheb_hi * l.lmax;
    const double theta = 0.5 * (bb + a), delta = 0.5 * (bb - a), sigma = theta / delta;
    double rho = 1.0 / sigma;
    const int N = l.n * m;
    const float* rin = b;
    if (!x_zero) {
        b_spmm(h, PK_SPMV, l.K, skern::SPMV_RESID, m, x, B.r, b, s);
        rin = B.r;
    }
    if (nu == 1) {
        b_asm(h, li, gm, m, rin, x, 1.0 / theta, x_zero ? 0.0 : 1.0, s);
        return;
    }
    b_asm(h, li, gm, m, rin, B.d, 1.0 / theta, 0.0, s);
    if (x_zero) {
        CK(cudaMemcpyAsync(x, B.d, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(B.r, b, sizeof(float) * N, cudaMemcpyDeviceToDevice, s));
    } else {
        axpby_l<float>(h, N, 1.0, B.d, 1.0, x, s);
    }
    for (int i = 1; i < nu; ++i) {
        b_spmm(h, PK_SPMV, l.K, skern::SPMV_RESID, m, B.d, B.r, B.r, s);    // r -= K d
        const double rho_new = 1.0 / (2.0 * sigma - rho);
        b_asm(h, li, gm, m, B.r, B.d, 2.0 * rho_new / delta, rho_new * rho, s);
        axpby_l<float>(h, N, 1.0, B.d, 1.0, x, s);
        rho = rho_new;
    }
}

void b_coarse(stokes_mg* h, int m, const float* b, float* e, cudaStream_t s) {
    const int n = h->nc;
    launch(h, -1, s, [&] { sbat::coarse_gemm(n, n + 1, m, h->Cinv, b, e, s); });
}

void b_hcycle(stokes_mg* h, int li, int gm, int m, const float* b, float* e, cudaStream_t s) {
    const int last = (int)h->L.size() - 1;
    if (li == last) { b_coarse(h, m, b, e, s); return; }
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    BatchLevel& C = h->bl[li + 1];
    const int nu = h->opts.nu_h;
    b_smooth(h, li, gm, m, b, e, true, nu, s);
    b_spmm(h, PK_SPMV, l.K, skern::SPMV_RESID, m, e, B.r, b, s);
    b_spmm(h, PK_TRANSFER, l.R, skern::SPMV_SET, m, B.r, C.b, nullptr, s);
    b_hcycle(h, li + 1, gm, m, C.b, C.e, s);
    b_spmm(h, PK_TRANSFER, l.P, skern::SPMV_ADD, m, C.e, e, nullptr, s);
    b_smooth(h, li, gm, m, b, e, false, nu, s);
}

void b_pcycle(stokes_mg* h, int li, int gm, int m, const float* b, float* e, cudaStream_t s) {
    const int last = (int)h->L.size() - 1;
    if (li == last) { b_coarse(h, m, b, e, s); return; }
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    if (!l.p_level) {
        b_hcycle(h, li, gm, m, b, e, s);
        for (int t = 1; t < h->opts.n_V; ++t) {
            b_spmm(h, PK_SPMV, l.K, skern::SPMV_RESID, m, e, B.t, b, s);
            b_hcycle(h, li, gm, m, B.t, B.u, s);
            axpby_l<float>(h, l.n * m, 1.0, B.u, 1.0, e, s);
        }
        return;
    }
    BatchLevel& C = h->bl[li + 1];
    const int nu = h->opts.nu_p;
    b_smooth(h, li, gm, m, b, e, true, nu, s);
    b_spmm(h, PK_SPMV, l.K, skern::SPMV_RESID, m, e, B.r, b, s);
    b_spmm(h, PK_TRANSFER, l.R, skern::SPMV_SET, m, B.r, C.b, nullptr, s);
    b_pcycle(h, li + 1, gm, m, C.b, C.e, s);
    b_spmm(h, PK_TRANSFER, l.P, skern::SPMV_ADD, m, C.e, e, nullptr, s);
    b_smooth(h, li, gm, m, b, e, false, nu, s);
}

// What gather_and_invert writes: the handle's stored form (factored saddle
// inverses or explicit inverses, in the handle's precision), the explicit
// inverse row-major in place of the gathered block (work), or explicit FP32
// inverses into l.inv32 (the batched path's operand).
enum InvOut { INV_STORE = 0, INV_BACK = 1, INV_EXPLICIT32 = 2 };
void gather_and_invert(stokes_mg* h, int li, double* work, int out, int* status, cudaStream_t s);

// The batched patch GEMM multiplies by explicit FP32 inverses.  A handle
// that stores factored saddle inverses builds them on first use (one gather
// and explicit saddle inversion per relaxed level, kept afterwards).
void ensure_explicit32(stokes_mg* h, cudaStream_t s) {
    const int nl = (int)h->L.size();
    for (int li = 0; li + 1 < nl; ++li) {
        DevLevel& l = h->L[li];
        if (l.inv32 || l.npatch == 0) continue;
        l.inv32 = halloc<float>(h, l.ninv32);
        double* work = palloc<double>(h->device, l.nsq, s);
        int* status = palloc<int>(h->device, l.npatch, s);
        CK(cudaMemsetAsync(status, 0, sizeof(int) * l.npatch, s));
        gather_and_invert(h, li, work, INV_EXPLICIT32, status, s);
        CK(cudaFreeAsync(work, s));
        CK(cudaFreeAsync(status, s));
    }
    CK(cudaStreamSynchronize(s));
}

// The 3xTF32 tensor-core GEMM reads each FP32 inverse as two arrays, its TF32
// part hi and the rest lo = a - hi, through their own tensor maps: built on
// the first 3xTF32 use and kept.
void ensure_split(stokes_mg* h, cudaStream_t s) {
    const int nl = (int)h->L.size();
    if ((int)h->tmaps_hi.size() == nl) return;
    h->inv_hi.assign(nl, nullptr);
    h->inv_lo.assign(nl, nullptr);
    std::vector<void*> mh(nl, nullptr), ml(nl, nullptr);
    for (int li = 0; li + 1 < nl; ++li) {
        DevLevel& l = h->L[li];
        h->inv_hi[li] = halloc<float>(h, l.ninv32);
        h->inv_lo[li] = halloc<float>(h, l.ninv32);
        mh[li] = halloc<unsigned char>(h, sbat::tmap_bytes(l.npatch));
        ml[li] = halloc<unsigned char>(h, sbat::tmap_bytes(l.npatch));
    }
    CK(cudaStreamSynchronize(h->s_up));      // new chunks are pool-ordered on s_up
    for (int li = 0; li + 1 < nl; ++li) {
        DevLevel& l = h->L[li];
        sbat::split_tf32(l.ninv32, l.inv32, h->inv_hi[li], h->inv_lo[li], s);
        CK(cudaGetLastError());
        sbat::build_tmaps(l.npatch, l.poff, l.ioff32, h->inv_hi[li], mh[li]);
        sbat::build_tmaps(l.npatch, l.poff, l.ioff32, h->inv_lo[li], ml[li]);
    }
    CK(cudaStreamSynchronize(s));
    h->tmaps_hi = mh;
    h->tmaps_lo = ml;
}

// interleaved work vectors of width m on every level (kept for later calls)
void ensure_batch(stokes_mg* h, int m) {
    if (!h->bstat_h) {
        CK(cudaHostAlloc((void**)&h->bstat_h, sizeof(int), cudaHostAllocMapped));
        *h->bstat_h = 0;
        CK(cudaHostGetDevicePointer((void**)&h->bstat_d, h->bstat_h, 0));
    }
    if (h->bm == m) return;
    const int nl = (int)h->L.size();
    h->bl.assign(nl, BatchLevel());
    for (int li = 0; li < nl; ++li) {
        const size_t N = (size_t)h->L[li].n * m;
        BatchLevel& B = h->bl[li];
        B.b = halloc<float>(h, N); B.e = halloc<float>(h, N); B.r = halloc<float>(h, N);
        B.d = halloc<float>(h, N); B.t = halloc<float>(h, N); B.u = halloc<float>(h, N);
        if (li + 1 < nl) B.Yb = halloc<float>(h, (size_t)h->L[li].nent * m);
    }
    // per-patch tensor maps over the FP32 inverses (the tensor-core TF32
    // path), built once per handle
    if (h->tmaps.empty()) {
        CK(cudaStreamSynchronize(h->s_up));
        ensure_explicit32(h, h->s_up);
        h->tmaps.assign(nl, nullptr);
        for (int li = 0; li + 1 < nl; ++li) h->tmaps[li] = halloc<unsigned char>(h, sbat::tmap_bytes(h->L[li].npatch));
        CK(cudaStreamSynchronize(h->s_up));
        for (int li = 0; li + 1 < nl; ++li) {
            DevLevel& l = h->L[li];
            sbat::build_tmaps(l.npatch, l.poff, l.ioff32, l.inv32, h->tmaps[li]);
        }
    }
    CK(cudaStreamSynchronize(h->s_up));      // new chunks are pool-ordered on s_up
    for (int i = 0; i < 2; ++i) {
        if (h->bgraph[i]) CK(cudaGraphExecDestroy(h->bgraph[i]));
        h->bgraph[i] = nullptr;
    }
    h->bm = m;
}

// Autotuner of the batched patch GEMM (one level, mode gm, width m).  The
// patches, sorted by size, are split into buckets of one kind (gemm_kind:
// the tensor cores for TF32 patches of more than 64 DoFs, the warp-level MMA
// otherwise) and one size class (128-row tiles for the tensor cores, 32-row
// groups for the warp kernel).  Each bucket's launch shape follows from its
// largest patch (pipeline stages and shared memory; for the warp kernel also
// the warps per CTA, of which the default and half are timed).  Adjacent
// buckets of one kind are then merged, left to right, while the merged launch
// is no slower than the two it replaces.  Every choice is timed on the
// level's own inverses (CUDA events, best of 3 after a warm-up).  A patch's
// arithmetic depends only on its kind, so the plan changes the time, never
// the result.
double time_gemm(stokes_mg* h, int li, int gm, int m, const stokes_mg::GemmPart& pt, const int* plist,
                 const float* X, cudaStream_t s) {
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    auto run = [&] {
        sbat::patch_gemm(gm, pt.kind, pt.nw, pt.count, plist ? plist + pt.off : nullptr, pt.hi, m, l.poff, l.pdofs,
                         l.ioff32, l.inv32, h->tmaps[li], split_map(h->tmaps_hi, li), split_map(h->tmaps_lo, li), X,
                         l.wt32, B.Yb, h->bstat_d, s);
        CK(cudaGetLastError());
    };
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    run();
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        CK(cudaEventRecord(e0, s));
        run();
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return 1e3 * best;
}

void tune_level(stokes_mg* h, int li, int gm, int m, cudaStream_t s) {
    using GemmPart = stokes_mg::GemmPart;
    DevLevel& l = h->L[li];
    BatchLevel& B = h->bl[li];
    const std::vector<int>& off = h->H.levels[li].patch_off;
    const int np = l.npatch;
    std::vector<int> idx(np), ns(np);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return off[a + 1] - off[a] < off[b + 1] - off[b]; });
    for (int i = 0; i < np; ++i) ns[i] = off[idx[i] + 1] - off[idx[i]];
    if ((int)h->bpsort.size() <= li) h->bpsort.resize(li + 1, nullptr);
    if (!h->bpsort[li]) {
        h->bpsort[li] = halloc<int>(h, np);
        CK(cudaStreamSynchronize(h->s_up));
        CK(cudaMemcpyAsync(h->bpsort[li], idx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
    }
    const int* plist = h->bpsort[li];
    float* X = B.u;                                       // zero input of the timing runs
    CK(cudaMemsetAsync(X, 0, sizeof(float) * (size_t)l.n * m, s));
    auto klass = [&](int n) {
        return sbat::gemm_kind(gm, n) == sbat::GEMM_KIND_TC ? 1000 + (n + 127) / 128 : (n + 31) / 32;
    };
    std::vector<GemmPart> parts;
    for (int i = 0; i < np;) {
        int j = i;
        while (j < np && klass(ns[j]) == klass(ns[i])) ++j;
        GemmPart pt;
        pt.kind = sbat::gemm_kind(gm, ns[i]);
        pt.off = i;
        pt.count = j - i;
        pt.lo = ns[i];
        pt.hi = ns[j - 1];
        parts.push_back(pt);
        i = j;
    }
    auto best_shape = [&](GemmPart& pt) {
        pt.nw = 0;
        pt.us = time_gemm(h, li, gm, m, pt, plist, X, s);
        if (pt.kind == sbat::GEMM_KIND_WARP) {
            const int nw0 = sbat::gemm_default_warps(pt.hi);
            if (nw0 > 1) {
                GemmPart half = pt;
                half.nw = (nw0 + 1) / 2;
                half.us = time_gemm(h, li, gm, m, half, plist, X, s);
                if (half.us < pt.us) pt = half;
            }
        }
    };
    for (auto& pt : parts) best_shape(pt);
    for (size_t i = 0; i + 1 < parts.size();) {
        if (parts[i].kind != parts[i + 1].kind) { ++i; continue; }
        GemmPart mg = parts[i];
        mg.count += parts[i + 1].count;
        mg.hi = parts[i + 1].hi;
        best_shape(mg);
        if (mg.us <= parts[i].us + parts[i + 1].us) {
            parts[i] = mg;
            parts.erase(parts.begin() + (long)i + 1);
        } else {
            ++i;
        }
    }
    // reference: one launch per kind over the whole level, default shape
    double single = 0;
    for (int kind : {sbat::GEMM_KIND_WARP, sbat::GEMM_KIND_TC}) {
        GemmPart all;
        all.kind = kind;
        for (const auto& pt : parts)
            if (pt.kind == kind) {
                if (all.count == 0) { all.off = pt.off; all.lo = pt.lo; }
                all.count += pt.count;
                all.hi = pt.hi;
            }
        if (all.count) single += time_gemm(h, li, gm, m, all, plist, X, s);
    }
    B.single_us[gm] = single;
    B.plan[gm] = parts;
}

// the plan of every relaxed level for mode gm at the current width: tuned,
// or (opts.batch_tune = 0) one launch per kind in size order
void ensure_plan(stokes_mg* h, int gm, int m, cudaStream_t s) {
    using GemmPart = stokes_mg::GemmPart;
    if (gm == sbat::GEMM_3XTF32) ensure_split(h, s);
    for (size_t li = 0; li + 1 < h->L.size(); ++li) {
        BatchLevel& B = h->bl[li];
        if (!B.plan[gm].empty()) continue;
        if (h->opts.batch_tune) {
            tune_level(h, (int)li, gm, m, s);
            continue;
        }
        const std::vector<int>& off = h->H.levels[li].patch_off;
        const int np = h->L[li].npatch;
        std::vector<int> idx(np);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return off[a + 1] - off[a] < off[b + 1] - off[b]; });
        if ((int)h->bpsort.size() <= (int)li) h->bpsort.resize(li + 1, nullptr);
        if (!h->bpsort[li]) {
            h->bpsort[li] = halloc<int>(h, np);
            CK(cudaStreamSynchronize(h->s_up));
            CK(cudaMemcpyAsync(h->bpsort[li], idx.data(), sizeof(int) * np, cudaMemcpyHostToDevice, s));
        }
        std::vector<GemmPart> parts;
        for (int i = 0; i < np;) {
            const int n0 = off[idx[i] + 1] - off[idx[i]], kind = sbat::gemm_kind(gm, n0);
            int j = i;
            while (j < np && sbat::gemm_kind(gm, off[idx[j] + 1] - off[idx[j]]) == kind) ++j;
            GemmPart pt;
            pt.kind = kind;
            pt.off = i;
            pt.count = j - i;
            pt.lo = n0;
            pt.hi = off[idx[j - 1] + 1] - off[idx[j - 1]];
            parts.push_back(pt);
            i = j;
        }
        B.plan[gm] = parts;
    }
    CK(cudaStreamSynchronize(s));
}

void capture_batched(stokes_mg* h, int gm, int m) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    long long before = h->launches;
    h->capturing = true;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        b_pcycle(h, 0, gm, m, h->bl[0].b, h->bl[0].e, cs);
    } catch (...) {
        cudaGraph_t dummy;
        cudaStreamEndCapture(cs, &dummy);
        h->capturing = false;
        cudaStreamDestroy(cs);
        throw;
    }
    CK(cudaStreamEndCapture(cs, &g));
    h->capturing = false;
    h->bgraph_launches[gm] = h->launches - before;
    h->launches = before;
    CK(cudaGraphInstantiate(&h->bgraph[gm], g, 0));
    CK(cudaGraphDestroy(g));
    CK(cudaStreamDestroy(cs));
}

// ---- reductions for FGMRES / Arnoldi (FP64, deterministic two-stage)
void mdot(stokes_mg* h, int n, int m, const double* V, long long ldv, const double* w, double* out, double* acc,
          bool sqrt_out, cudaStream_t s, const KrylovWS* ws = nullptr) {
    double* partial = ws ? ws->partial : h->partial;
    unsigned int* ticket = ws ? ws->ticket : h->ticket;
    launch(h, -1, s, [&] {
        skern::mdot_fused(n, m, V, ldv, w, partial, ticket, out, acc, sqrt_out ? 1 : 0, s);
    });
}

void maxpy_l(stokes_mg* h, int n, int m, const double* V, long long ldv, const double* hh, double sign, double* w,
             cudaStream_t s) {
    launch(h, -1, s, [&] { skern::maxpy<<<grid_for(n), 256, 0, s>>>(n, m, V, ldv, hh, sign, w); });
}

// Orthogonalise w (length n) against V[0..m-1] by classical Gram-Schmidt
// applied twice, then normalise it: hcoef[0..m-1] receives the summed
// coefficients, hn[0] = ||w|| before the normalisation (the new Hessenberg
// entry).  Three launches: the first pass's dots; its update fused with the
// second pass's dots and ||w||^2; the second update with the scaling.
// h2 holds m + 1 values.
void cgs2(stokes_mg* h, int n, int m, const double* V, double* w, double* hcoef, double* h2, double* hn, cudaStream_t s,
          const KrylovWS* ws = nullptr) {
    double* partial = ws ? ws->partial : h->partial;
    unsigned int* ticket = ws ? ws->ticket : h->ticket;
    mdot(h, n, m, V, n, w, hcoef, nullptr, false, s, ws);
    launch(h, -1, s, [&] {
        skern::maxpy_mdot(n, m, V, n, hcoef, w, partial, ticket, h2, hcoef, s);
    });
    launch(h, -1, s, [&] { skern::maxpy_normalise<<<grid_for(n), 256, 0, s>>>(n, m, V, n, h2, h2 + m, w, hn); });
}

double d2h_scalar(stokes_mg* h, const double* d, cudaStream_t s) {
    CK(cudaMemcpyAsync(h->pinned, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return h->pinned[0];
}

// Arnoldi lambda_max on level li from v0 (device, FP64): all steps run on
// the device without host round trips; the (m+1) x m Hessenberg matrix is
// then read once, truncated at the first breakdown H[j+1][j] <= 1e-14
// |H[j][j]|, and its eigenvalues found on the host (a 15 x 15 problem).
// Launch `steps` Arnoldi steps on M_l^{-1} K_l from v0 on stream s (no host
// round trip) and queue the copy of the (m+1) x m Hessenberg matrix into
// H_host (pinned); returns m.  Uses the FGMRES basis V as workspace, so
// launches on one stream run one level after another.
int arnoldi_launch(stokes_mg* h, int li, const double* v0, int steps, double* Hs, double* H_host, cudaStream_t s,
                   const KrylovWS* ws = nullptr) {
    DevLevel& l = h->L[li];
    const int n = l.n;
    const int m = std::min(steps, std::min(n, skern::HESS_MAX - 1));
    double* V = ws ? ws->V : h->V;
    double* hh = ws ? ws->h : h->h;
    double* yy = ws ? ws->y : h->y;
    double* hn = ws ? ws->hn : h->hn;
    launch(h, -1, s, [&] { skern::fill_vec<double><<<1, 256, 0, s>>>((long long)(m + 1) * m, 0.0, Hs); });
    mdot(h, n, 1, v0, n, v0, hn, nullptr, true, s, ws);
    launch(h, -1, s, [&] { skern::scale_by_inv<<<grid_for(n), 256, 0, s>>>(n, v0, hn, V); });
    // the operator M^{-1} K is applied in the precision of the smoother that
    // the estimate serves (FP32 K and inverses in mixed mode); the basis and
    // its orthogonalisation stay FP64
    const bool f32 = h->opts.precision == STOKES_MIXED && (l.inv32 || l.fac32) && l.K.v32 && l.t32 && l.u32;
    for (int j = 0; j < m; ++j) {
        double* w = V + (long long)(j + 1) * n;
        if (f32) {
            launch(h, -1, s, [&] { skern::convert_vec<float, double><<<grid_for(n), 256, 0, s>>>(n, V + (long long)j * n, l.t32); });
            spmv<float>(h, PK_SPMV, l.K, skern::SPMV_SET, l.t32, l.u32, nullptr, s);
            asm_apply<float>(h, l, l.u32, l.t32, 1.0, 0.0, s);
            launch(h, -1, s, [&] { skern::convert_vec<double, float><<<grid_for(n), 256, 0, s>>>(n, l.t32, w); });
        } else {
            spmv<double>(h, PK_SPMV, l.K, skern::SPMV_SET, V + (long long)j * n, l.t64, nullptr, s);
            asm_apply<double>(h, l, l.t64, w, 1.0, 0.0, s);
        }
        cgs2(h, n, j + 1, V, w, hh, yy, hn, s, ws);
        launch(h, -1, s, [&] { skern::arnoldi_store<<<1, 1, 0, s>>>(j, m, Hs, hh, hn); });
    }
    CK(cudaMemcpyAsync(H_host, Hs, sizeof(double) * (m + 1) * m, cudaMemcpyDeviceToHost, s));
    return m;
}

// Largest real Ritz value from a Hessenberg matrix read back by
// arnoldi_launch, truncated at the first breakdown H[j+1][j] <= 1e-14 |H[j][j]|
// (a 15 x 15 eigenproblem, solved on the host).
double arnoldi_finish(const double* H, int m) {
    int used = m;
    for (int j = 0; j < m; ++j) {
        const double sub = H[(size_t)(j + 1) * m + j], dj = H[(size_t)j * m + j];
        if (!std::isfinite(sub) || !std::isfinite(dj)) throw StokesError(STOKES_ENONFINITE, "non-finite Arnoldi entry");
        if (std::fabs(sub) <= 1e-14 * std::fabs(dj) + 1e-300) { used = j + 1; break; }
    }
    skern::cplx A[skern::HESS_MAX][skern::HESS_MAX], cr[skern::HESS_MAX], sr[skern::HESS_MAX];
    double out[2];
    skern::hessenberg_eig_core(used, m, H, out, A, cr, sr);
    return out[0];
}

double arnoldi_lmax(stokes_mg* h, int li, const double* v0, int steps, cudaStream_t s) {
    double* Hs = h->Hh;
    double* Hh = h->pinned_H;
    const int m = arnoldi_launch(h, li, v0, steps, Hs, Hh, s);
    CK(cudaStreamSynchronize(s));
    return arnoldi_finish(Hh, m);
}

// SplitMix64 start vector (the same counter-based definition as the tests'
// generator): value i of stream `st` in [-1, 1).
__global__ void splitmix_uniform(int n, unsigned long long seed, unsigned long long st, double* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long z = seed + (st * (1ULL << 32) + (unsigned long long)i + 1ULL) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        out[i] = (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    }
}

using Precond = std::function<void(const double*, double*, cudaStream_t)>;

// FGMRES(restart) for K x = b right-preconditioned by M (Sec. 4), x0 = 0;
// rscr is an n-vector of scratch.
int fgmres_op(stokes_mg* h, const DevCSR& K, int n, double* rscr, const Precond& M, const double* b, double* x,
              double tol, int* its_out, double* rel_out, cudaStream_t s) {
    const int m = h->restart;
    launch(h, -1, s, [&] { skern::fill_vec<double><<<grid_for(n), 256, 0, s>>>(n, 0.0, x); });
    mdot(h, n, 1, b, n, b, h->hn, nullptr, true, s);
    const double beta0 = d2h_scalar(h, h->hn, s);
    if (!std::isfinite(beta0)) throw StokesError(STOKES_ENONFINITE, "non-finite right-hand side");
    int its = 0;
    double rel = 0.0;
    if (beta0 == 0.0) {
        if (its_out) *its_out = 0;
        if (rel_out) *rel_out = 0.0;
        return STOKES_OK;
    }
    double* r = rscr;
    const double* rcur = b;
    double beta = beta0;
    bool converged = false;
    std::vector<double> g0(m + 1, 0.0);
    while (its < h->opts.maxit) {
        // V[0] = r / beta, g = (beta, 0, ...)
        g0.assign(m + 1, 0.0);
        g0[0] = beta;
        CK(cudaMemcpyAsync(h->g, g0.data(), sizeof(double) * (m + 1), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(h->scal, &g0[0], sizeof(double), cudaMemcpyHostToDevice, s));
        launch(h, -1, s, [&] { skern::scale_by_inv<<<grid_for(n), 256, 0, s>>>(n, rcur, h->scal, h->V); });
        CK(cudaStreamSynchronize(s));   // g0 is a host temporary
        int jend = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = h->V + (long long)j * n;
            double* zj = h->Z + (long long)j * n;
            double* w = h->V + (long long)(j + 1) * n;
            M(vj, zj, s);
            spmv<double>(h, PK_SPMV, K, skern::SPMV_SET, zj, w, nullptr, s);
            cgs2(h, n, j + 1, h->V, w, h->h, h->y, h->hn, s);
            launch(h, -1, s, [&] {
                skern::fgmres_givens<<<1, 1, 0, s>>>(j, m, h->Hh, h->h, h->hn, h->cs, h->sn, h->g, h->resid);
            });
            const double res = d2h_scalar(h, h->resid, s);
            ++its;
            jend = j + 1;
            if (!std::isfinite(res)) throw StokesError(STOKES_ENONFINITE, "non-finite FGMRES residual");
            rel = res / beta0;
            if (res <= tol * beta0) { converged = true; break; }
            if (its >= h->opts.maxit) break;
        }
        launch(h, -1, s, [&] { skern::fgmres_backsolve<<<1, 1, 0, s>>>(jend, m, h->Hh, h->g, h->y); });
        maxpy_l(h, n, jend, h->Z, n, h->y, 1.0, x, s);
        if (converged) break;
        spmv<double>(h, PK_SPMV, K, skern::SPMV_RESID, x, r, b, s);
        mdot(h, n, 1, r, n, r, h->hn, nullptr, true, s);
        beta = d2h_scalar(h, h->hn, s);
        rel = beta / beta0;
        if (beta <= tol * beta0) { converged = true; break; }
        rcur = r;
    }
    check_sa_status(h, s);
    if (its_out) *its_out = its;
    if (rel_out) *rel_out = rel;
    return converged ? STOKES_OK : STOKES_ENOTCONVERGED;
}

void fbf_apply(stokes_mg* h, const double* r, double* z, cudaStream_t s);

// FGMRES-phMG on the finest level (Sec. 4), or FGMRES-FBF(phMG) in FBF mode
int fgmres(stokes_mg* h, const double* b, double* x, double tol, int* its_out, double* rel_out, cudaStream_t s) {
    if (h->fbf) {
        FbfData& F = *h->fbf;
        return fgmres_op(h, F.S0d.K, F.nS, F.r, [h](const double* v, double* z, cudaStream_t st) { fbf_apply(h, v, z, st); },
                         b, x, tol, its_out, rel_out, s);
    }
    DevLevel& l0 = h->L[0];
    const int n = l0.n, prec = h->opts.precision;
    return fgmres_op(h, l0.K, n, l0.t64,
                     [h, n, prec](const double* v, double* z, cudaStream_t st) {
                         CK(cudaMemcpyAsync(h->vin, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
                         vcycle_run(h, prec, st);
                         CK(cudaMemcpyAsync(z, h->vout, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
                     },
                     b, x, tol, its_out, rel_out, s);
}

// P^-1 r of Eq. fbf on the Stokes free DoFs (velocity components blocked,
// then pressure): a = A~^-1 r_u, z_p = S~^-1 (r_p - B a),
// z_u = A~^-1 (r_u - B^T z_p).  A~^-1 is the scalar phMG V-cycle on every
// velocity component; B a and B^T z_p come from the Stokes K applied to
// (a, 0) and (0, z_p); S~^-1 is the block-diagonal -nu_e M_p,e^-1.
void fbf_apply(stokes_mg* h, const double* r, double* z, cudaStream_t s) {
    FbfData& F = *h->fbf;
    const int nu = F.nu, nS = F.nS, nvf = F.nvf, d = F.S0.d, np = nS - nu, prec = h->opts.precision;
    auto vcycles = [&](const double* in, double* out) {
        for (int c = 0; c < d; ++c) {
            CK(cudaMemcpyAsync(h->vin, in + (size_t)c * nvf, sizeof(double) * nvf, cudaMemcpyDeviceToDevice, s));
            vcycle_run(h, prec, s);
            CK(cudaMemcpyAsync(out + (size_t)c * nvf, h->vout, sizeof(double) * nvf, cudaMemcpyDeviceToDevice, s));
        }
    };
    vcycles(r, F.a);
    CK(cudaMemcpyAsync(F.t, F.a, sizeof(double) * nu, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(F.t + nu, 0, sizeof(double) * np, s));
    spmv<double>(h, PK_SPMV, F.S0d.K, skern::SPMV_SET, F.t, F.w, nullptr, s);      // w_p = B a
    axpby_l<double>(h, np, 1.0, r + nu, -1.0, F.w + nu, s);                         // w_p = r_p - B a
    launch(h, -1, s, [&] {
        skern::block_mass_inverse<<<grid_for((long long)F.ncell * F.nbq), 256, 0, s>>>(F.ncell, F.nbq, F.qcell, F.minv,
                                                                                      F.scale, F.w + nu, z + nu);
    });
    CK(cudaMemsetAsync(F.t, 0, sizeof(double) * nu, s));
    CK(cudaMemcpyAsync(F.t + nu, z + nu, sizeof(double) * np, cudaMemcpyDeviceToDevice, s));
    spmv<double>(h, PK_SPMV, F.S0d.K, skern::SPMV_SET, F.t, F.w, nullptr, s);      // w_u = B^T z_p
    axpby_l<double>(h, nu, 1.0, r, -1.0, F.w, s);                                   // w_u = r_u - B^T z_p
    vcycles(F.w, z);
}

// FBF data on the device: the Stokes operator, work vectors, and S~^-1 as
// a reference inverse mass matrix with one scale per cell
void setup_fbf(stokes_mg* h, cudaStream_t s) {
    FbfData& F = *h->fbf;
    const sfem::Level& S0 = F.S0;
    const sfem::Mesh& m = h->H.meshes[S0.mesh_index];
    F.a = halloc<double>(h, F.nu);
    F.t = halloc<double>(h, F.nS);
    F.w = halloc<double>(h, F.nS);
    F.r = halloc<double>(h, F.nS);
    const int d = m.d;
    F.ncell = m.nc;
    F.nbq = S0.Q.nb;
    // inverse of the reference mass matrix of the pressure degree (Gauss-Jordan, partial pivoting)
    const int nb = F.nbq;
    std::vector<double> Mr = sfem::reference_mass(d, S0.k - 1), inv((size_t)nb * nb, 0.0);
    for (int i = 0; i < nb; ++i) inv[(size_t)i * nb + i] = 1.0;
    for (int c = 0; c < nb; ++c) {
        int piv = c;
        for (int r = c + 1; r < nb; ++r)
            if (std::fabs(Mr[(size_t)r * nb + c]) > std::fabs(Mr[(size_t)piv * nb + c])) piv = r;
        for (int j = 0; j < nb; ++j) {
            std::swap(Mr[(size_t)c * nb + j], Mr[(size_t)piv * nb + j]);
            std::swap(inv[(size_t)c * nb + j], inv[(size_t)piv * nb + j]);
        }
        const double p = Mr[(size_t)c * nb + c];
        if (p == 0.0) throw StokesError(STOKES_ESINGULAR, "singular reference pressure mass matrix");
        for (int j = 0; j < nb; ++j) { Mr[(size_t)c * nb + j] /= p; inv[(size_t)c * nb + j] /= p; }
        for (int r = 0; r < nb; ++r) {
            if (r == c) continue;
            const double f = Mr[(size_t)r * nb + c];
            if (f == 0.0) continue;
            for (int j = 0; j < nb; ++j) {
                Mr[(size_t)r * nb + j] -= f * Mr[(size_t)c * nb + j];
                inv[(size_t)r * nb + j] -= f * inv[(size_t)c * nb + j];
            }
        }
    }
    F.minv = hupload(h, inv, s);
    // scale_e = -nu_e / |det J_e|: M_p,e = |det J_e| M_ref on an affine cell
    std::vector<double> scale(m.nc);
    for (int e = 0; e < m.nc; ++e) {
        const int* C = &m.C[(size_t)e * (d + 1)];
        double J[9];
        for (int a = 0; a < d; ++a)
            for (int c = 0; c < d; ++c) J[c * d + a] = m.X[(size_t)C[a + 1] * d + c] - m.X[(size_t)C[0] * d + c];
        const double det = d == 2 ? J[0] * J[3] - J[1] * J[2]
                                  : J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                                        J[2] * (J[3] * J[7] - J[4] * J[6]);
        const double nue = S0.nu_cells.empty() ? 1.0 : S0.nu_cells[e];
        scale[e] = -nue / std::fabs(det);
    }
    F.scale = hupload(h, scale, s);
    F.qcell = hupload(h, S0.Q.cell_nodes, s);
}

// ---------------------------------------------------------------- setup --
void upload_assembly_inputs(stokes_mg* h, int li, bool want32, cudaStream_t s);

// Operator part of a level (its CSR, or the inputs of the device assembly)
// and the level's work vectors.
void upload_level_operator(stokes_mg* h, int li, bool want32, cudaStream_t s) {
    const sfem::Level& HL = h->H.levels[li];
    DevLevel& l = h->L[li];
    l.n = HL.n_free;
    l.p_level = HL.p_level;
    double tt = host_ms();
    if (HL.host_matrices) {
        l.K = upload_csr(h, HL.K, want32, s);
    } else {
        upload_assembly_inputs(h, li, want32, s);
    }
    trace("upload K", li, tt);
    l.b64 = halloc<double>(h, l.n); l.e64 = halloc<double>(h, l.n); l.r64 = halloc<double>(h, l.n);
    l.d64 = halloc<double>(h, l.n); l.t64 = halloc<double>(h, l.n); l.u64 = halloc<double>(h, l.n);
    if (want32) {
        l.b32 = halloc<float>(h, l.n); l.e32 = halloc<float>(h, l.n); l.r32 = halloc<float>(h, l.n);
        l.d32 = halloc<float>(h, l.n); l.t32 = halloc<float>(h, l.n); l.u32 = halloc<float>(h, l.n);
    }
}

// Patch part of a relaxed level: index sets, offsets of the dense blocks and
// inverses, partition-of-unity weights and the DoF -> slot map.
void upload_level_patches(stokes_mg* h, int li, bool want32, cudaStream_t s) {
    const sfem::Level& HL = h->H.levels[li];
    DevLevel& l = h->L[li];
    double tt = host_ms();
    const bool last = li + 1 == (int)h->H.levels.size();
    if (!last) {
        l.npatch = (int)HL.patch_off.size() - 1;
        l.nent = HL.patch_dofs.size();
        std::vector<long long> moff(l.npatch + 1, 0), o64(l.npatch + 1, 0), o32(l.npatch + 1, 0);
        l.maxn = 0;
        for (int p = 0; p < l.npatch; ++p) {
            const long long n = HL.patch_off[p + 1] - HL.patch_off[p];
            l.maxn = std::max<int>(l.maxn, (int)n);
            moff[p + 1] = moff[p] + n * n;
            o64[p + 1] = o64[p] + ((n + 1) & ~1LL) * n;
            o32[p + 1] = o32[p] + ((n + 3) & ~3LL) * n;
        }
        l.nsq = moff[l.npatch];
        l.ninv64 = o64[l.npatch];
        l.ninv32 = o32[l.npatch];
        trace("patch offsets (host)", li, tt);
        l.poff = hupload(h, HL.patch_off, s);
        l.pdofs = hupload(h, HL.patch_dofs, s);
        l.pnv = hupload(h, HL.patch_nv, s);
        trace("patch lists uploaded", li, tt);
        std::vector<long long> scoff(l.npatch + 1, 0);
        for (int p = 0; p < l.npatch; ++p) {
            const long long sc = skern::saddle_scratch(HL.d, HL.patch_off[p + 1] - HL.patch_off[p], HL.patch_nv[p]);
            if (sc <= skern::SADDLE_SMEM_MAX_DOUBLES) {
                l.saddle_smem = std::max(l.saddle_smem, sc);
                l.saddle_smem_fac = std::max(l.saddle_smem_fac, skern::saddle_scratch_factored(
                                                                    HL.d, HL.patch_off[p + 1] - HL.patch_off[p],
                                                                    HL.patch_nv[p]));
                scoff[p + 1] = scoff[p];
            }
            else
                scoff[p + 1] = scoff[p] + std::max(sc, skern::saddle_scratch_factored(
                                                           HL.d, HL.patch_off[p + 1] - HL.patch_off[p], HL.patch_nv[p],
                                                           false));
        }
        l.saddle_global = scoff[l.npatch];
        l.scoff = hupload(h, scoff, s);
        l.moff = hupload(h, moff, s);
        l.ioff64 = hupload(h, o64, s);
        l.ioff32 = hupload(h, o32, s);
        // partition of unity W_i = diag(1/m_j) and the DoF -> slot map
        trace("block offsets uploaded", li, tt);
        // slots of every DoF in increasing order (the pull scatter's order)
        // and the weights W_i = 1 / multiplicity, built on the device
        l.wt64 = halloc<double>(h, l.n);
        l.soff = halloc<int>(h, (size_t)l.n + 1);
        l.sidx = halloc<int>(h, l.nent);
        {
            const int n = l.n;
            int* scr = palloc<int>(h->device, 2 * (size_t)n + (n + 1023) / 1024 + 2, s);
            int *cnt = scr, *cur = scr + n, *stmp = scr + 2 * n;
            CK(cudaMemsetAsync(scr, 0, sizeof(int) * 2 * (size_t)n, s));
            launch(h, -1, s, [&] { skern::slot_count<<<grid_for(l.nent), 256, 0, s>>>(l.nent, l.pdofs, cnt); });
            launch(h, -1, s, [&] { sasm::scan_rows(cnt, n, l.soff, stmp, s); });
            launch(h, -1, s, [&] { skern::slot_fill<<<grid_for(l.nent), 256, 0, s>>>(l.nent, l.pdofs, l.soff, cur, l.sidx); });
            launch(h, -1, s, [&] { skern::slot_sort<<<grid_for(n), 256, 0, s>>>(n, l.soff, l.sidx, l.wt64); });
            CK(cudaFreeAsync(scr, s));
        }
        trace("patch maps", li, tt);
        tt = host_ms();
        l.Y64 = halloc<double>(h, l.nent);
        // the stored inverses: the factored saddle form for the saddle-block
        // solver, explicit otherwise; FP32 on MIXED handles (the V-cycle and
        // the lambda_max estimate run in FP32 there), FP64 on FP64 handles
        l.factored = h->opts.patch_solver == 0;
        if (l.factored) {
            std::vector<long long> f64(l.npatch + 1, 0), f32(l.npatch + 1, 0);
            l.sa_xs = l.maxn;
            for (int p = 0; p < l.npatch; ++p) {
                const int n = HL.patch_off[p + 1] - HL.patch_off[p], nv = HL.patch_nv[p];
                const int np = n - HL.d * nv;
                f64[p + 1] = f64[p] + skern::saddle_factor_len(HL.d, n, nv, 2);
                f32[p + 1] = f32[p] + skern::saddle_factor_len(HL.d, n, nv, 4);
                l.sa_ws64 = std::max<long long>(l.sa_ws64, (long long)((HL.d * nv + 1) & ~1) * np);
                l.sa_ws32 = std::max<long long>(l.sa_ws32, (long long)((HL.d * nv + 3) & ~3) * np);
            }
            l.nfac64 = f64[l.npatch];
            l.nfac32 = f32[l.npatch];
            if (skern::saddle_apply_smem(8, 2, 0, l.sa_xs) > skern::SADDLE_APPLY_SMEM_MAX)
                throw StokesError(STOKES_EUNSUPPORTED, "patch too large for the saddle apply's shared memory");
            // one process-wide upper bound (never lowered)
            CK(cudaFuncSetAttribute(skern::saddle_apply_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)skern::SADDLE_APPLY_SMEM_MAX));
            CK(cudaFuncSetAttribute(skern::saddle_apply_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)skern::SADDLE_APPLY_SMEM_MAX));
            CK(cudaFuncSetAttribute(skern::saddle_apply_bulk_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)skern::SADDLE_APPLY_SMEM_MAX));
            CK(cudaFuncSetAttribute(skern::saddle_apply_bulk_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)skern::SADDLE_APPLY_SMEM_MAX));
            // the bulk-copy apply, with L^-1 stored as its packed upper
            // triangle, when the level's largest packed block fits in shared
            // memory with room for at least two CTAs per SM
            {
                const int eb = want32 ? 4 : 8, vec = 16 / eb;
                long long mb = 0;
                std::vector<long long> fp(l.npatch + 1, 0);
                for (int p = 0; p < l.npatch; ++p) {
                    const long long len = skern::saddle_factor_len(HL.d, HL.patch_off[p + 1] - HL.patch_off[p],
                                                                   HL.patch_nv[p], vec, 1);
                    fp[p + 1] = fp[p] + len;
                    mb = std::max(mb, len);
                }
                const long long buf = (mb * eb + 127) & ~127LL;
                const size_t smem = skern::saddle_apply_bulk_smem((int)std::min<long long>(buf, 1 << 30), eb, l.sa_xs);
                if (buf > 0 && smem <= skern::SADDLE_APPLY_SMEM_MAX / 2 && !std::getenv("STOKES_NO_BULK_APPLY")) {
                    l.sa_buf = (int)buf;
                    l.fac_packed = true;
                    (want32 ? f32 : f64) = fp;
                    (want32 ? l.nfac32 : l.nfac64) = fp[l.npatch];
                }
                if (!h->sa_status) {
                    h->sa_status = halloc<int>(h, 1);
                    CK(cudaMemsetAsync(h->sa_status, 0, sizeof(int), s));
                }
            }
            if (want32) { l.foff32 = hupload(h, f32, s); l.fac32 = halloc<float>(h, l.nfac32); }
            else { l.foff64 = hupload(h, f64, s); l.fac64 = halloc<double>(h, l.nfac64); }
        } else if (!want32) {
            l.inv64 = halloc<double>(h, l.ninv64);
        }
        if (want32) {
            l.wt32 = halloc<float>(h, l.n);
            skern::convert_vec<float, double><<<grid_for(l.n), 256, 0, s>>>(l.n, l.wt64, l.wt32);
            CK(cudaGetLastError());
            l.Y32 = halloc<float>(h, l.nent);
            if (!l.factored) l.inv32 = halloc<float>(h, l.ninv32);
        }
    }
    trace("patch uploads + allocs", li, tt);
}

// Mesh, DoF maps, adjacency and reference tensors of a level whose K is
// assembled on the device; K's arrays are sized by an upper bound on the
// row lengths (incident cells times nodes per cell).
void upload_assembly_inputs_lv(stokes_mg* h, const sfem::Level& HL, DevLevel& l, bool want32, cudaStream_t s);
void upload_assembly_inputs(stokes_mg* h, int li, bool want32, cudaStream_t s) {
    upload_assembly_inputs_lv(h, h->H.levels[li], h->L[li], want32, s);
}
void upload_assembly_inputs_lv(stokes_mg* h, const sfem::Level& HL, DevLevel& l, bool want32, cudaStream_t s) {
    const sfem::Mesh& mesh = h->H.meshes[HL.mesh_index];
    const int nm = (int)h->H.meshes.size();
    if ((int)h->mesh_X.size() != nm) { h->mesh_X.assign(nm, nullptr); h->mesh_C.assign(nm, nullptr); }
    if (!h->mesh_X[HL.mesh_index]) {
        h->mesh_X[HL.mesh_index] = hupload(h, mesh.X, s);
        h->mesh_C[HL.mesh_index] = hupload(h, mesh.C, s);
    }
    sasm::AsmMesh& a = l.am;
    a.d = HL.d;
    a.nc = mesh.nc;
    a.nb = HL.V.nb;
    a.nq = HL.Q.nb;
    a.nV = HL.V.n;
    a.nQ = HL.nQ;
    a.nVf = HL.nVf;
    a.X = h->mesh_X[HL.mesh_index];
    a.C = h->mesh_C[HL.mesh_index];
    a.vcell = hupload(h, HL.V.cell_nodes, s);
    a.qcell = hupload(h, HL.Q.cell_nodes, s);
    a.vfree = hupload(h, HL.vfree, s);
    std::vector<int> vrow(HL.nVf);
    for (int i = 0; i < HL.V.n; ++i)
        if (HL.vfree[i] >= 0) vrow[HL.vfree[i]] = i;
    a.vrow = hupload(h, vrow, s);
    // node -> cell incidence lists from the cell-node maps, on the device
    {
        const long long mv = (long long)mesh.nc * a.nb, mq = (long long)mesh.nc * a.nq;
        const int nmax = std::max(HL.V.n, HL.nQ);
        int* voff = halloc<int>(h, HL.V.n + 1);
        int* vadj = halloc<int>(h, std::max<long long>(mv, 1));
        int* qoff = halloc<int>(h, HL.nQ + 1);
        int* qadj = halloc<int>(h, std::max<long long>(mq, 1));
        int* cnt = halloc<int>(h, nmax);
        int* cur = halloc<int>(h, nmax);
        int* tmp = halloc<int>(h, (nmax + 1023) / 1024 + 2);
        launch(h, -1, s, [&] { sasm::node_cells(a.vcell, mv, HL.V.n, voff, vadj, cnt, cur, tmp, s); });
        launch(h, -1, s, [&] { sasm::node_cells(a.qcell, mq, HL.nQ, qoff, qadj, cnt, cur, tmp, s); });
        h->launches += 10;               // six kernels per list
        a.voff = voff;
        a.vadj = vadj;
        a.qoff = qoff;
        a.qadj = qadj;
    }
    a.nu = HL.nu_cells.empty() ? nullptr : hupload(h, HL.nu_cells, s);
    a.S = hupload(h, HL.RT.S, s);
    a.Cq = hupload(h, HL.RT.Cq, s);
    a.M = hupload(h, HL.RT.M, s);
    l.cellgeo = halloc<double>(h, (size_t)mesh.nc * sasm::CG_STRIDE);
    a.cg = l.cellgeo;
    sasm::set_list_caps(a, HL.max_cells);
    // entries: a velocity row of a node in c cells has at most c (nb + nq),
    // a pressure row at most d c nb; the incidences sum to nc nb and nc nq
    const long long bound = (long long)HL.d * mesh.nc * a.nb * (a.nb + a.nq) + (long long)HL.d * mesh.nc * a.nq * a.nb;
    // the CSR's row pointers and column indices are 32-bit
    if (bound > INT32_MAX)
        throw StokesError(STOKES_EUNSUPPORTED, "level operator beyond 2^31 - 1 entries (32-bit CSR indices)");
    const int n = HL.n_free;
    DevCSR& K = l.K;
    K.nr = K.nc = n;
    K.nnz = bound;                       // exact count read back once setup has synchronised
    K.rp = halloc<int>(h, n + 1);
    K.ci = halloc<int>(h, bound);
    K.v64 = halloc<double>(h, bound);
    K.v32 = want32 ? halloc<float>(h, bound) : nullptr;
    K.lanes = 4;                         // rows of ~25-120 entries (choose_lanes after assembly)
    l.asm_len = halloc<int>(h, n);
    l.asm_tmp = halloc<int>(h, (n + 1023) / 1024 + 2);
    l.asm_status = halloc<int>(h, 1);
    CK(cudaMemsetAsync(l.asm_status, 0, sizeof(int), s));
    l.dev_asm = true;
}

// K of a device-assembled level: row lengths, scan, values (stream s)
void assemble_dev(stokes_mg* h, DevLevel& l, cudaStream_t s);
void assemble_on_device(stokes_mg* h, int li, cudaStream_t s) {
    DevLevel& l = h->L[li];
    if (!l.am.vcell) return;        // the FBF velocity level 0 is filtered, not assembled
    assemble_dev(h, l, s);
}
void assemble_dev(stokes_mg* h, DevLevel& l, cudaStream_t s) {
    if (!l.dev_asm) return;
    const int n = l.K.nr;
    launch(h, -1, s, [&] { sasm::cell_geometry(l.am, l.cellgeo, s); });
    launch(h, -1, s, [&] { sasm::row_lengths(l.am, l.asm_len, l.asm_status, s); });
    launch(h, -1, s, [&] { sasm::scan_rows(l.asm_len, n, l.K.rp, l.asm_tmp, s); });
    launch(h, -1, s, [&] { sasm::fill_rows(l.am, l.K.rp, l.K.ci, l.K.v64, l.asm_status, s); });
    if (l.K.v32)
        launch(h, -1, s, [&] {
            skern::convert_vec<float, double><<<grid_for(l.K.nnz), 256, 0, s>>>((int)l.K.nnz, l.K.v64, l.K.v32);
        });
}

// exact nnz of the device-assembled operators (after the setup stream synchronised)

// FBF: level 0's operator.  The SV Stokes K of the finest mesh is assembled
// on the device (FbfData::S0d, also the outer FGMRES operator and the input
// of the matrix-free load); the scalar velocity level's K is its leading
// (component-0 velocity) block, filtered on the device.  Uploads on s_up,
// kernels on `target` (after the uploads).
void fbf_level0_operator(stokes_mg* h, bool want32, cudaStream_t target) {
    FbfData& F = *h->fbf;
    const sfem::Level& HL = h->H.levels[0];
    DevLevel& l = h->L[0];
    l.n = HL.n_free;
    l.p_level = HL.p_level;
    l.b64 = halloc<double>(h, l.n); l.e64 = halloc<double>(h, l.n); l.r64 = halloc<double>(h, l.n);
    l.d64 = halloc<double>(h, l.n); l.t64 = halloc<double>(h, l.n); l.u64 = halloc<double>(h, l.n);
    if (want32) {
        l.b32 = halloc<float>(h, l.n); l.e32 = halloc<float>(h, l.n); l.r32 = halloc<float>(h, l.n);
        l.d32 = halloc<float>(h, l.n); l.t32 = halloc<float>(h, l.n); l.u32 = halloc<float>(h, l.n);
    }
    upload_assembly_inputs_lv(h, F.S0, F.S0d, false, h->s_up);
    const int n = l.n;
    const long long bound = F.S0d.K.nnz;
    DevCSR& K = l.K;
    K.nr = K.nc = n;
    K.nnz = bound;
    K.rp = halloc<int>(h, n + 1);
    K.ci = halloc<int>(h, bound);
    K.v64 = halloc<double>(h, bound);
    K.v32 = want32 ? halloc<float>(h, bound) : nullptr;
    K.lanes = 4;
    l.asm_len = halloc<int>(h, n);
    l.asm_tmp = halloc<int>(h, (n + 1023) / 1024 + 2);
    l.asm_status = halloc<int>(h, 1);
    CK(cudaMemsetAsync(l.asm_status, 0, sizeof(int), h->s_up));
    l.dev_asm = true;                   // nnz and lanes are fixed up with the assembled levels
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, h->s_up));
    CK(cudaStreamWaitEvent(target, ev, 0));
    CK(cudaEventDestroy(ev));
}

void fbf_level0_kernels(stokes_mg* h, cudaStream_t s) {
    FbfData& F = *h->fbf;
    DevLevel& l = h->L[0];
    const DevCSR& A = F.S0d.K;
    const int n = l.n;
    assemble_dev(h, F.S0d, s);
    launch(h, -1, s, [&] { skern::csr_block_count<<<grid_for(n), 256, 0, s>>>(n, n, A.rp, A.ci, l.asm_len); });
    launch(h, -1, s, [&] { sasm::scan_rows(l.asm_len, n, l.K.rp, l.asm_tmp, s); });
    launch(h, -1, s, [&] {
        skern::csr_block_fill<<<grid_for(n), 256, 0, s>>>(n, n, A.rp, A.ci, A.v64, l.K.rp, l.K.ci, l.K.v64, l.K.v32);
    });
}

void upload_transfers(stokes_mg* h, int li, bool want32, cudaStream_t s) {
    const sfem::Level& HL = h->H.levels[li];
    DevLevel& l = h->L[li];
    if (l.dev_transfer) return;          // built on the device
    l.P = upload_csr(h, HL.P, want32, s);
    l.R = upload_csr(h, HL.R, want32, s);
}

// mesh data the device transfers read (vertex coordinates, cells, parents)
void ensure_mesh_on_device(stokes_mg* h, int mi, cudaStream_t s) {
    const int nm = (int)h->H.meshes.size();
    if ((int)h->mesh_X.size() != nm) { h->mesh_X.assign(nm, nullptr); h->mesh_C.assign(nm, nullptr); }
    if ((int)h->mesh_parent.size() != nm) h->mesh_parent.assign(nm, nullptr);
    if (!h->mesh_X[mi]) {
        h->mesh_X[mi] = hupload(h, h->H.meshes[mi].X, s);
        h->mesh_C[mi] = hupload(h, h->H.meshes[mi].C, s);
    }
    if (mi + 1 < nm && !h->mesh_parent[mi]) h->mesh_parent[mi] = hupload(h, h->H.parents[mi], s);
}

// P_l (coarse level l + 1 -> fine level l, Sec. 3.1) and R_l = P_l^T built
// on the device from the two levels' DoF maps (uploaded on s_up before the
// launch: the fine level's assembly inputs, the coarse level's cell nodes
// and free map).  Host uploads happen here, on the calling (host) thread;
// `launch_on` queues the kernels.  The exact entry counts are read back by
// finish_setup.
void build_transfer_dev(stokes_mg* h, int li, bool want32, const std::function<void(std::function<void()>)>& launch_on) {
    const sfem::Level& F = h->H.levels[li];
    const sfem::Level& C = h->H.levels[li + 1];
    DevLevel& lf = h->L[li];
    DevLevel& lc = h->L[li + 1];
    const cudaStream_t su = h->s_up;
    const int d = F.d;
    const bool nested = F.mesh_index != C.mesh_index;
    const sfem::RefElement& rVf = sfem::reference_element(d, F.k);
    const sfem::RefElement& rQf = sfem::reference_element(d, F.k - 1);
    const sfem::RefElement& rVc = sfem::reference_element(d, C.k);
    const sfem::RefElement& rQc = sfem::reference_element(d, C.k - 1);
    if (rVc.nb > sasm::INTERP_MAX_NB || rQc.nb > sasm::INTERP_MAX_NB)
        throw StokesError(STOKES_EUNSUPPORTED, "coarse element too large for the device transfer");
    sasm::InterpGeom gV, gQ;
    gV.d = gQ.d = d;
    gV.nested = gQ.nested = nested ? 1 : 0;
    if (!nested) {
        // coarse basis at the fine lattice points of the same cell
        auto table = [&](const sfem::RefElement& rf, const sfem::RefElement& rc) {
            std::vector<double> t((size_t)rf.nb * rc.nb);
            for (int l = 0; l < rf.nb; ++l) {
                double xi[3] = {0, 0, 0};
                for (int a = 0; a < d; ++a) xi[a] = (double)rf.alpha[l][a + 1] / rf.k;
                rc.eval(xi, t.data() + (size_t)l * rc.nb);
            }
            return t;
        };
        gV.tab = hupload(h, table(rVf, rVc), su);
        gQ.tab = hupload(h, table(rQf, rQc), su);
    } else {
        ensure_mesh_on_device(h, F.mesh_index, su);
        ensure_mesh_on_device(h, C.mesh_index, su);
        auto fill = [&](sasm::InterpGeom& g, const sfem::RefElement& rf, const sfem::RefElement& rc) {
            g.parent = h->mesh_parent[F.mesh_index];
            g.Xf = h->mesh_X[F.mesh_index]; g.Cf = h->mesh_C[F.mesh_index];
            g.Xc = h->mesh_X[C.mesh_index]; g.Cc = h->mesh_C[C.mesh_index];
            g.kf = rf.k;
            std::vector<int> al((size_t)rf.nb * 4), mo((size_t)rc.nm * 3);
            for (int l = 0; l < rf.nb; ++l)
                for (int a = 0; a < 4; ++a) al[(size_t)l * 4 + a] = rf.alpha[l][a];
            for (int m = 0; m < rc.nm; ++m)
                for (int a = 0; a < 3; ++a) mo[(size_t)m * 3 + a] = rc.mono[m][a];
            g.alpha_f = hupload(h, al, su);
            g.nm = rc.nm;
            g.mono = hupload(h, mo, su);
            g.coef = hupload(h, rc.coef, su);
        };
        fill(gV, rVf, rVc);
        fill(gQ, rQf, rQc);
    }
    sasm::InterpSpace fV, fQ, cV, cQ;
    fV.nb = F.V.nb; fV.cell = lf.am.vcell; fV.off = lf.am.voff; fV.adj = lf.am.vadj; fV.free = lf.am.vfree;
    fQ.nb = F.Q.nb; fQ.cell = lf.am.qcell; fQ.off = lf.am.qoff; fQ.adj = lf.am.qadj; fQ.free = nullptr;
    cV.nb = C.V.nb; cV.cell = lc.am.vcell; cV.free = lc.am.vfree;
    cQ.nb = C.Q.nb; cQ.cell = lc.am.qcell; cQ.free = nullptr;
    const int nVf = F.nVf, nQf = F.nQ, nr = F.n_free, nrR = C.n_free;
    const long long ubP = (long long)d * nVf * cV.nb + (long long)nQf * cQ.nb;
    if (ubP > INT32_MAX)
        throw StokesError(STOKES_EUNSUPPORTED, "transfer beyond 2^31 - 1 entries (32-bit CSR indices)");
    DevCSR& P = lf.P;
    DevCSR& R = lf.R;
    P.nr = nr; P.nc = nrR; P.nnz = ubP;
    R.nr = nrR; R.nc = nr; R.nnz = ubP;
    P.rp = halloc<int>(h, nr + 1); P.ci = halloc<int>(h, ubP); P.v64 = halloc<double>(h, ubP);
    R.rp = halloc<int>(h, nrR + 1); R.ci = halloc<int>(h, ubP); R.v64 = halloc<double>(h, ubP);
    if (want32) { P.v32 = halloc<float>(h, ubP); R.v32 = halloc<float>(h, ubP); }
    // rows of ~1-6 (P) and ~10-60 (R) entries (lanes fixed again at finish)
    P.lanes = R.lanes = 4;
    lf.dev_transfer = true;
    const int* vrow = lf.am.vrow;
    launch_on([h, gV, gQ, fV, fQ, cV, cQ, nVf, nQf, nr, nrR, d, ubP, vrow, P, R, want32, nVf_c = C.nVf] {
        const cudaStream_t s = h->s_tr;
        int* cntV = palloc<int>(h->device, std::max(nVf, 1), s);
        int* colV = palloc<int>(h->device, std::max<long long>((long long)nVf * cV.nb, 1), s);
        double* valV = palloc<double>(h->device, std::max<long long>((long long)nVf * cV.nb, 1), s);
        int* cntQ = palloc<int>(h->device, std::max(nQf, 1), s);
        int* colQ = palloc<int>(h->device, std::max<long long>((long long)nQf * cQ.nb, 1), s);
        double* valQ = palloc<double>(h->device, std::max<long long>((long long)nQf * cQ.nb, 1), s);
        int* len = palloc<int>(h->device, std::max(nr, nrR) + 1, s);
        int* tmp = palloc<int>(h->device, (std::max(nr, nrR) + 1023) / 1024 + 2, s);
        int* cur = palloc<int>(h->device, std::max(nrR, 1), s);
        launch(h, -1, s, [&] { sasm::interp_rows(gV, fV, cV, nVf, vrow, cntV, colV, valV, s); });
        launch(h, -1, s, [&] { sasm::interp_rows(gQ, fQ, cQ, nQf, nullptr, cntQ, colQ, valQ, s); });
        launch(h, -1, s, [&] { sasm::interp_lengths(d, nVf, nQf, cntV, cntQ, len, s); });
        launch(h, -1, s, [&] { sasm::scan_rows(len, nr, P.rp, tmp, s); });
        launch(h, -1, s, [&] {
            sasm::interp_fill(d, nVf, nQf, nVf_c, cV.nb, cQ.nb, cntV, colV, valV, cntQ, colQ, valQ, P.rp, P.ci, P.v64, s);
        });
        launch(h, -1, s, [&] { sasm::transpose_count(nr, P.rp, P.ci, nrR, len, s); });
        launch(h, -1, s, [&] { sasm::scan_rows(len, nrR, R.rp, tmp, s); });
        launch(h, -1, s, [&] { sasm::transpose_fill(nr, P.rp, P.ci, P.v64, nrR, R.rp, cur, R.ci, R.v64, s); });
        launch(h, -1, s, [&] { sasm::sort_rows(nrR, R.rp, R.ci, R.v64, s); });
        if (want32) {
            launch(h, -1, s, [&] { sasm::to_float(ubP, P.v64, P.v32, s); });
            launch(h, -1, s, [&] { sasm::to_float(ubP, R.v64, R.v32, s); });
        }
        for (void* x : {(void*)cntV, (void*)colV, (void*)valV, (void*)cntQ, (void*)colQ, (void*)valQ, (void*)len,
                        (void*)tmp, (void*)cur})
            CK(cudaFreeAsync(x, s));
    });
}

// gather K_i and invert every patch of level li; work receives the
// row-major inverses (sum n_i^2 doubles) when keep != nullptr.
// whether level li's factored inverses are computed straight from its CSR
// operator (every patch inverted in shared memory, with room for its DoF list)
bool fused_factor(const stokes_mg* h, const DevLevel& l) {
    return h->opts.patch_solver == 0 && !l.inv64 && !l.inv32 && l.saddle_global == 0 && l.saddle_smem > 0 &&
           l.saddle_smem_fac + (l.maxn + 1) / 2 <= skern::SADDLE_SMEM_MAX_DOUBLES;
}

void gather_and_invert(stokes_mg* h, int li, double* work, int out, int* status, cudaStream_t s) {
    DevLevel& l = h->L[li];
    if (l.npatch == 0) return;
    const bool fused = out == INV_STORE && fused_factor(h, l);
    if (!fused) {
        launch(h, -1, s, [&] { skern::fill_vec<double><<<grid_for(l.nsq), 256, 0, s>>>(l.nsq, 0.0, work); });
        launch(h, -1, s, [&] {
            skern::patch_gather<<<l.npatch, 256, l.maxn * sizeof(int), s>>>(l.npatch, l.poff, l.pdofs, l.moff, l.K.rp,
                                                                           l.K.ci, l.K.v64, work);
        });
    }
    const bool store = out == INV_STORE;
    double* i64 = store ? l.inv64 : nullptr;
    float* i32 = store || out == INV_EXPLICIT32 ? l.inv32 : nullptr;
    const int back = out == INV_BACK ? 1 : 0;
    if (h->opts.patch_solver == 0) {
        // saddle block inverse (default)
        const int d = h->dim;
        double* f64 = store ? l.fac64 : nullptr;
        float* f32 = store ? l.fac32 : nullptr;
        if (l.saddle_smem > 0) {
            const bool fac_only = !i64 && !i32 && !back;
            const long long sd_off = fac_only ? l.saddle_smem_fac : l.saddle_smem;
            const size_t smem = (size_t)(sd_off + (fused ? (l.maxn + 1) / 2 : 0)) * sizeof(double);
            // one upper bound for every level (levels launch from one thread
            // onto different streams)
            CK(cudaFuncSetAttribute(skern::saddle_inverse_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(skern::SADDLE_SMEM_MAX_DOUBLES * sizeof(double))));
            launch(h, PK_GJ, s, [&] {
                skern::saddle_inverse_smem<<<l.npatch, 256, smem, s>>>(
                    l.npatch, d, l.poff, l.pnv, l.moff, fused ? nullptr : work, l.ioff64, i64, l.ioff32, i32, l.foff64, f64,
                    l.foff32, f32, back, l.fac_packed ? 1 : 0, skern::SADDLE_SMEM_MAX_DOUBLES, l.pdofs, l.K.rp, l.K.ci,
                    l.K.v64, (int)sd_off, status);
            });
        }
        if (l.saddle_global > 0) {
            // scratch of the patches too large for shared memory, from the
            // stream-ordered pool (freed on the same stream, no host wait)
            double* scr = palloc<double>(h->device, l.saddle_global, s);
            launch(h, PK_GJ, s, [&] {
                skern::saddle_inverse_global<<<l.npatch, 256, 0, s>>>(l.npatch, d, l.poff, l.pnv, l.moff, work, l.ioff64, i64,
                                                                      l.ioff32, i32, l.foff64, f64, l.foff32, f32, back,
                                                                      l.fac_packed ? 1 : 0, skern::SADDLE_SMEM_MAX_DOUBLES,
                                                                      l.scoff, scr, status);
            });
            CK(cudaFreeAsync(scr, s));
        }
        return;
    }
    const int nsm = std::min(l.maxn, skern::GJ_SMEM_MAX_N);
    const size_t smem = (size_t)nsm * nsm * sizeof(double) + nsm * sizeof(double) + nsm * sizeof(int) + 64;
    {
        const int gmax = skern::GJ_SMEM_MAX_N;
        CK(cudaFuncSetAttribute(skern::gj_inverse_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)gmax * gmax * sizeof(double) + gmax * sizeof(double) + gmax * sizeof(int) + 64)));
    }
    launch(h, PK_GJ, s, [&] {
        skern::gj_inverse_smem<<<l.npatch, 256, smem, s>>>(l.npatch, l.poff, l.moff, work, i64 ? l.ioff64 : nullptr, i64,
                                                           i32 ? l.ioff32 : nullptr, i32, status, 0);
    });
    if (l.maxn > skern::GJ_SMEM_MAX_N) {
        int* ipiv = palloc<int>(h->device, l.nent, s);
        double* col = palloc<double>(h->device, l.nent, s);
        launch(h, PK_GJ, s, [&] {
            skern::gj_inverse_global<<<l.npatch, 512, 0, s>>>(l.npatch, l.poff, l.moff, work, i64 ? l.ioff64 : nullptr, i64,
                                                              i32 ? l.ioff32 : nullptr, i32, status, ipiv, col);
        });
        CK(cudaFreeAsync(ipiv, s));
        CK(cudaFreeAsync(col, s));
    }
}

// Launch the gather + inversion of level li on stream s without waiting;
// the workspace and status array stay in h->pending until finish_setup.
void launch_patches(stokes_mg* h, int li, cudaStream_t s) {
    DevLevel& l = h->L[li];
    if (l.npatch == 0) return;
    PendingPatches pp;
    pp.level = li;
    pp.work = fused_factor(h, l) ? nullptr : palloc<double>(h->device, l.nsq, s);
    pp.status = palloc<int>(h->device, l.npatch, s);
    pp.stream = s;   // freed on the same stream after finish_setup synchronised it
    h->pending.push_back(pp);
    CK(cudaMemsetAsync(pp.status, 0, sizeof(int) * l.npatch, s));
    gather_and_invert(h, li, pp.work, INV_STORE, pp.status, s);
}

void free_pending(stokes_mg* h) {
    for (auto& pp : h->pending) {
        if (pp.work) cudaFreeAsync(pp.work, pp.stream);
        cudaFreeAsync(pp.status, pp.stream);
    }
    h->pending.clear();
}

// Wait for every launched patch inversion and report the first zero pivot.

// Bordered coarse matrix (zero-mean pressure constraint, Sec. 2) inverted in
// place on stream s (no wait): by one thread-block cluster when its rows fit
// in the cluster's shared memory, else by one Gauss-Jordan step per pivot.
void upload_coarse(stokes_mg* h, cudaStream_t su) {
    const sfem::Level& C = h->H.levels.back();
    const int n = C.n_free, nb = n + 1;
    h->nc = n;
    std::vector<double> A((size_t)nb * nb, 0.0);
    for (int r = 0; r < n; ++r)
        for (int p = C.K.rp[r]; p < C.K.rp[r + 1]; ++p) A[(size_t)r * nb + C.K.ci[p]] = C.K.v[p];
    // border with c_j = int psi_j on the pressure DoFs (zero-mean pressure, Sec. 2)
    for (int q = 0; q < C.nQ; ++q) {
        const int r = C.d * C.nVf + q;
        A[(size_t)r * nb + n] = C.pint[q];
        A[(size_t)n * nb + r] = C.pint[q];
    }
    // no pressure (the scalar velocity hierarchy of FBF): [A 0; 0 1], whose
    // inverse applied to (b, 0) is (A^-1 b, 0)
    if (C.nQ == 0) A[(size_t)n * nb + n] = 1.0;
    h->Cinv = hupload(h, A, su);
    h->c_ipiv = dalloc<int>(nb);
    h->c_colk = dalloc<double>(nb);
    h->c_status = dalloc<int>(1);
    CK(cudaMemsetAsync(h->c_status, 0, sizeof(int), su));
}

// can one cluster of GJC_CTAS CTAs run gj_cluster_panel with this much
// dynamic shared memory on this device?
bool cluster_panel_ok(stokes_mg* h, size_t smem) {
    if (cudaFuncSetAttribute(skern::gj_cluster_panel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(skern::gj_cluster_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = skern::GJC_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(skern::GJC_CTAS);
    cfg.blockDim = dim3(skern::GJC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, skern::gj_cluster_panel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nclusters > 0;
}

void launch_coarse(stokes_mg* h, cudaStream_t s) {
    const int nb = h->nc + 1;
    // blocked Gauss-Jordan: the pivots of a panel of B columns on one cluster
    // of 16 CTAs (each holding its share of the rows of the panel), then the
    // panel's row swaps and the rank-B update of every other column on all
    // SMs (32 x 32 tiles).  The per-pivot cluster work is rows/16 x B, so the
    // pivot chain costs little more than its two cluster barriers per pivot.
    const int B = skern::GJB_MAX_B;
    const size_t psmem = (size_t)skern::gj_cluster_panel_smem_doubles(nb, B) * sizeof(double);
    const bool clus = cluster_panel_ok(h, psmem);
    if (!clus) CK(cudaFuncSetAttribute(skern::gj_block_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    const int Bb = [&] {
        int b = B;
        while (!clus && b > 1 && skern::gj_block_panel_smem(nb, b) > 200 * 1024) b >>= 1;
        return b;
    }();
    if (clus || skern::gj_block_panel_smem(nb, Bb) <= 200 * 1024) {
        double* Pk = palloc<double>(h->device, (size_t)nb * Bb, s);
        double* Yb = palloc<double>(h->device, (size_t)nb * Bb, s);
        const dim3 ug((nb + 31) / 32, (nb + 31) / 32);
        for (int k0 = 0; k0 < nb; k0 += Bb) {
            const int b = std::min(Bb, nb - k0);
            if (clus) {
                launch(h, -1, s, [&] {
                    cudaLaunchConfig_t cfg = {};
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeClusterDimension;
                    attr[0].val.clusterDim.x = skern::GJC_CTAS;
                    attr[0].val.clusterDim.y = 1;
                    attr[0].val.clusterDim.z = 1;
                    cfg.gridDim = dim3(skern::GJC_CTAS);
                    cfg.blockDim = dim3(skern::GJC_THREADS);
                    cfg.dynamicSmemBytes = psmem;
                    cfg.stream = s;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    CK(cudaLaunchKernelEx(&cfg, skern::gj_cluster_panel, nb, k0, b, h->Cinv, h->c_ipiv, Pk,
                                          h->c_status));
                });
            } else {
                launch(h, -1, s, [&] {
                    skern::gj_block_panel<<<1, skern::GJB_THREADS, skern::gj_block_panel_smem(nb, b), s>>>(
                        nb, k0, b, h->Cinv, h->c_ipiv, Pk, h->c_status);
                });
            }
            launch(h, -1, s, [&] { skern::gj_block_swap<<<(nb + 255) / 256, 256, 0, s>>>(nb, k0, b, h->Cinv, h->c_ipiv, Yb); });
            launch(h, -1, s, [&] { skern::gj_block_update<<<ug, 256, 0, s>>>(nb, k0, b, h->Cinv, Pk, Yb); });
        }
        launch(h, -1, s, [&] { skern::gj_unpivot_rows<<<grid_for(nb), 256, 0, s>>>(nb, h->Cinv, h->c_ipiv); });
        CK(cudaFreeAsync(Pk, s));
        CK(cudaFreeAsync(Yb, s));
        return;
    }
    const long long tot = (long long)nb * nb;
    const int egrid = (int)std::min<long long>((tot + 255) / 256, 152LL * 8);
    for (int k = 0; k < nb; ++k) {
        launch(h, -1, s, [&] { skern::gj_step_pivot<<<1, 256, 0, s>>>(nb, k, h->Cinv, h->c_ipiv, h->c_colk, h->c_status); });
        launch(h, -1, s, [&] { skern::gj_step_eliminate<<<egrid, 256, 0, s>>>(nb, k, h->Cinv, h->c_colk); });
    }
    launch(h, -1, s, [&] { skern::gj_unpivot_rows<<<grid_for(nb), 256, 0, s>>>(nb, h->Cinv, h->c_ipiv); });
}

void free_coarse_ws(stokes_mg* h) {
    if (h->c_ipiv) cudaFree(h->c_ipiv);
    if (h->c_colk) cudaFree(h->c_colk);
    if (h->c_status) cudaFree(h->c_status);
    h->c_ipiv = nullptr;
    h->c_colk = nullptr;
    h->c_status = nullptr;
}


// pinned room for finish_setup's readback (allocated while the device still
// works on level 0, off the critical path)
void alloc_readback(stokes_mg* h) {
    size_t n = 8 + 4 * (h->L.size() + 1);
    for (const auto& l : h->L) n += (size_t)std::max(l.npatch, 0);
    if (n <= h->n_rb) return;
    if (h->pinned_rb) CK(cudaFreeHost(h->pinned_rb));
    CK(cudaMallocHost((void**)&h->pinned_rb, sizeof(int) * n));
    h->n_rb = n;
}

// What the host still needs from the setup kernels, with one wait: every
// setup stream is joined into s, the patch statuses, the assembly statuses
// and sizes, the transfer sizes and the coarse and apply statuses are copied
// into pinned memory on s, and s is synchronised once.  The checks then run
// in that order: patches, assembly, transfers, coarse factorisation, apply.
void finish_setup(stokes_mg* h, cudaStream_t s) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    std::vector<cudaStream_t> ss(h->s_lvl.begin(), h->s_lvl.end());
    ss.push_back(h->s_tr);
    ss.push_back(h->s_coarse);
    ss.push_back(h->s_up);
    for (cudaStream_t x : ss)
        if (x && x != s) {
            CK(cudaEventRecord(ev, x));
            CK(cudaStreamWaitEvent(s, ev, 0));
        }
    CK(cudaEventDestroy(ev));
    alloc_readback(h);
    int* rb = h->pinned_rb;
    size_t o = 0;
    auto get = [&](const int* d, size_t n) {
        if (o + n > h->n_rb) throw StokesError(STOKES_ECUDA, "internal: setup readback overflow");
        CK(cudaMemcpyAsync(rb + o, d, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        const size_t at = o;
        o += n;
        return at;
    };
    std::vector<size_t> at_pp;
    for (auto& pp : h->pending) at_pp.push_back(get(pp.status, (size_t)h->L[pp.level].npatch));
    std::vector<DevLevel*> asm_lv;
    if (h->fbf && h->fbf->S0d.dev_asm) asm_lv.push_back(&h->fbf->S0d);
    for (auto& l : h->L)
        if (l.dev_asm) asm_lv.push_back(&l);
    std::vector<size_t> at_asm;
    for (DevLevel* l : asm_lv) {
        at_asm.push_back(get(l->asm_status, 1));
        get(l->K.rp + l->K.nr, 1);
    }
    std::vector<size_t> at_tr(h->L.size(), 0);
    for (size_t li = 0; li + 1 < h->L.size(); ++li)
        if (h->L[li].dev_transfer) at_tr[li] = get(h->L[li].P.rp + h->L[li].P.nr, 1);
    const size_t at_c = h->c_status ? get(h->c_status, 1) : 0;
    const size_t at_sa = h->sa_status ? get(h->sa_status, 1) : 0;
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < h->pending.size(); ++i) {
        const auto& pp = h->pending[i];
        const int np = h->L[pp.level].npatch;
        for (int p = 0; p < np; ++p)
            if (rb[at_pp[i] + p] != 0) {
                h->st.singular_patch = pp.level * (1 << 24) + p;
                throw StokesError(STOKES_ESINGULAR, "zero pivot in patch " + std::to_string(p) + " of level " +
                                                        std::to_string(pp.level));
            }
    }
    free_pending(h);
    for (size_t i = 0; i < asm_lv.size(); ++i) {
        DevLevel& l = *asm_lv[i];
        if (rb[at_asm[i]] != 0) throw StokesError(STOKES_EUNSUPPORTED, "a node has more than 1024 neighbours");
        l.K.nnz = rb[at_asm[i] + 1];
        l.K.lanes = choose_lanes(l.K);
    }
    for (size_t li = 0; li + 1 < h->L.size(); ++li) {
        DevLevel& l = h->L[li];
        if (!l.dev_transfer) continue;
        l.P.nnz = l.R.nnz = rb[at_tr[li]];
        l.P.lanes = choose_lanes(l.P);
        l.R.lanes = choose_lanes(l.R);
    }
    const int cst = h->c_status ? rb[at_c] : 0;
    free_coarse_ws(h);
    if (cst != 0) {
        h->st.singular_patch = -2;
        throw StokesError(STOKES_ESINGULAR, "zero pivot in the coarse bordered LU");
    }
    if (h->sa_status && rb[at_sa] != 0)
        throw StokesError(STOKES_ECUDA, "a patch-apply CTA gave up waiting for its bulk copy (bounded wait)");
}

void setup_solve_buffers(stokes_mg* h, cudaStream_t s) {
    const sfem::Level& F = finest_stokes(h);
    const int d = F.d;
    if (F.host_matrices) {
        h->Mv = upload_csr(h, F.Mv, false, s);
        h->KfD = upload_csr(h, F.KfD, false, s);
    }
    std::vector<int> rows(d * F.nVf);
    std::vector<int> vrow(F.nVf);
    for (int i = 0; i < F.V.n; ++i)
        if (F.vfree[i] >= 0) vrow[F.vfree[i]] = i;
    for (int c = 0; c < d; ++c)
        for (int f = 0; f < F.nVf; ++f) rows[c * F.nVf + f] = c * F.V.n + vrow[f];
    h->vel_rows = hupload(h, rows, s);
    h->F = halloc<double>(h, (size_t)d * F.V.n);
    h->gzero = halloc<double>(h, (size_t)d * F.V.n);
    CK(cudaMemsetAsync(h->gzero, 0, sizeof(double) * d * F.V.n, s));
    h->bvec = halloc<double>(h, F.n_free);
    h->xvec = halloc<double>(h, F.n_free);
    std::vector<double> ones(F.nQ, 1.0);
    h->ones = hupload(h, ones, s);
    h->pint = hupload(h, F.pint, s);
    h->pint_sum = 0;
    for (double v : F.pint) h->pint_sum += v;
}

// Arnoldi scratch of relaxed level li >= 1 (its own stream and buffers)
void alloc_level_krylov(stokes_mg* h, int li, cudaStream_t s) {
    const int n = h->L[li].n;
    if ((int)h->kws.size() < (int)h->L.size()) h->kws.resize(h->L.size());
    KrylovWS& w = h->kws[li];
    w.V = halloc<double>(h, (size_t)skern::HESS_MAX * n);
    w.v0 = halloc<double>(h, n);
    w.h = halloc<double>(h, skern::HESS_MAX + 1);
    w.y = halloc<double>(h, skern::HESS_MAX + 1);
    w.hn = halloc<double>(h, 2);
    w.partial = halloc<double>(h, (size_t)skern::MDOT_BLOCKS * 32);
    w.ticket = halloc<unsigned int>(h, 1);
    CK(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned int), s));
}

// FGMRES / Arnoldi buffers sized by the finest level
void alloc_krylov(stokes_mg* h, cudaStream_t s) {
    const int n0 = h->L[0].n;
    const int nK = h->fbf ? std::max(n0, h->fbf->nS) : n0;     // FBF: FGMRES runs on the Stokes system
    const int m = h->restart;
    const int basis = std::max(m + 1, skern::HESS_MAX + 1);
    h->V = halloc<double>(h, (size_t)basis * nK);
    h->Z = halloc<double>(h, (size_t)m * nK);
    h->Hh = halloc<double>(h, (size_t)(basis + 1) * basis);
    h->cs = halloc<double>(h, basis);
    h->sn = halloc<double>(h, basis);
    h->g = halloc<double>(h, basis + 1);
    h->y = halloc<double>(h, basis + 1);
    h->h = halloc<double>(h, basis + 1);
    h->hn = halloc<double>(h, 2);
    h->resid = halloc<double>(h, 2);
    h->scal = halloc<double>(h, 4);
    h->partial_blocks = skern::MDOT_BLOCKS;
    h->partial = halloc<double>(h, (size_t)h->partial_blocks * 32);
    h->ticket = halloc<unsigned int>(h, 1);
    CK(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), s));
    h->vin = halloc<double>(h, n0);
    h->vout = halloc<double>(h, n0);
    h->v0buf = halloc<double>(h, n0);
    CK(cudaMallocHost((void**)&h->pinned, 64));
}

// Hessenberg matrices of the lambda_max estimates: one device and one pinned
// host slot per level (allocated with the first level that reaches setup)
void alloc_hess(stokes_mg* h, cudaStream_t s) {
    h->Hlev = halloc<double>(h, (size_t)STOKES_MAX_LEVELS * skern::HESS_MAX * skern::HESS_MAX);
    CK(cudaMallocHost((void**)&h->pinned_H, sizeof(double) * (STOKES_MAX_LEVELS + 1) * skern::HESS_MAX * skern::HESS_MAX));
}

void fill_stats(stokes_mg* h) {
    stokes_mg_stats& st = h->st;
    st.n_levels = (int)h->H.levels.size();
    st.dim = h->dim;
    st.family = h->family;
    st.k = h->k;
    for (int i = 0; i < st.n_levels; ++i) {
        const sfem::Level& HL = h->H.levels[i];
        st.n_free[i] = HL.n_free;
        st.degree[i] = HL.k;
        st.level_family[i] = HL.family;
        st.mesh_index[i] = HL.mesh_index;
        st.is_p_level[i] = HL.p_level ? 1 : 0;
        st.nnz[i] = (!HL.host_matrices && i < (int)h->L.size()) ? h->L[i].K.nnz : HL.K.nnz();
        const int np = HL.patch_off.empty() ? 0 : (int)HL.patch_off.size() - 1;
        long long sq = 0;
        int mx = 0;
        for (int p = 0; p < np; ++p) {
            const long long n = HL.patch_off[p + 1] - HL.patch_off[p];
            sq += n * n;
            mx = std::max<int>(mx, (int)n);
        }
        st.n_patches[i] = np;
        st.max_patch[i] = mx;
        st.patch_entries[i] = sq;
        st.lmax[i] = i < (int)h->L.size() ? h->L[i].lmax : 0.0;
    }
    st.n_vel_nodes = finest_stokes(h).V.n;
    st.n_pres_nodes = finest_stokes(h).nQ;
}

int fail(const StokesError& e) {
    g_last_error = e.what();
    return e.code;
}

template <typename F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const StokesError& e) {
        return fail(e);
    } catch (const std::invalid_argument& e) {
        g_last_error = e.what();
        return STOKES_EINVAL;
    } catch (const std::length_error& e) {         // a size beyond the 32-bit indices of the host build
        g_last_error = e.what();
        return STOKES_EUNSUPPORTED;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return STOKES_EOOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return STOKES_EINVAL;
    }
}

void require(bool c, const char* msg) {
    if (!c) throw StokesError(STOKES_EINVAL, msg);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(const stokes_mg* h) {
        require(!h->host_only, "the handle was built with host_only: no device data");
        const int dev = h->device;
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// temporary FP32/FP64 conversions for the per-step entry points
struct Tmp32 {
    float* p = nullptr;
    explicit Tmp32(size_t n) { p = dalloc<float>(n); }
    ~Tmp32() { cudaFree(p); }
};

}  // namespace

// =================================================================== C ABI
extern "C" {

const char* stokes_last_error(void) { return g_last_error.c_str(); }

void stokes_mg_default_opts(stokes_mg_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hierarchy = STOKES_HIER_GRADUAL;
    o->nu_p = o->nu_h = o->n_V = 1;
    o->eig_steps = 15;
    o->eig_seed = 0;
    o->cheb_lo = 0.1;
    o->cheb_hi = 1.1;
    o->precision = STOKES_FP64;
    o->restart = 30;
    o->maxit = 1000;
    o->use_graph = 1;
    o->batch_tune = 1;
}

namespace {
int setup_impl(const stokes_mesh* coarse, int n_refine, int barycentric_finest, int family, int k,
               const stokes_mg_opts* opts, const double* nu_cell, void* stream, stokes_mg_t* out, bool fbf_mode) {
    g_last_error.clear();
    if (!out) { g_last_error = "out is NULL"; return STOKES_EINVAL; }
    *out = nullptr;
    auto h = std::make_unique<stokes_mg>();
    std::memset(&h->st, 0, sizeof(h->st));
    h->st.singular_patch = -1;
    int rc = guarded([&] {
        const double t0 = host_ms();
        require(coarse && coarse->verts && coarse->cells, "mesh is NULL");
        require(coarse->dim == 2 || coarse->dim == 3, "dim must be 2 or 3");
        require(coarse->n_verts > 0 && coarse->n_cells > 0, "empty mesh");
        require(n_refine >= 0 && n_refine <= 8, "n_refine out of range");
        require(family == STOKES_TH || family == STOKES_SV, "unknown family");
        require(family == STOKES_TH || barycentric_finest, "Scott-Vogelius needs the barycentric finest mesh");
        require(k >= 2 && k <= 10, "k must be in [2, 10]");
        if (opts) h->opts = *opts; else stokes_mg_default_opts(&h->opts);
        stokes_mg_opts& o = h->opts;
        require(o.nu_p >= 1 && o.nu_h >= 1 && o.n_V >= 1 && o.nu_p <= 16 && o.nu_h <= 16 && o.n_V <= 16, "bad sweep counts");
        require(o.restart >= 1 && o.restart <= 31, "restart must be in [1, 31]");
        require(o.eig_steps >= 1 && o.eig_steps <= 15, "eig_steps must be in [1, 15]");
        require(o.precision == STOKES_FP64 || o.precision == STOKES_MIXED, "bad precision");
        require(o.cheb_hi > o.cheb_lo && o.cheb_lo > 0, "bad Chebyshev interval");
        require(o.patch_solver == 0 || o.patch_solver == 1, "patch_solver must be 0 (saddle block) or 1 (Gauss-Jordan)");
        if (!o.host_only) CK(cudaGetDevice(&h->device));
        if (!o.host_only) mark(h.get(), "setup start", (cudaStream_t)stream);
        for (int kk = 0; kk < 5; ++kk) h->prof[kk].on = (o.prof_mask >> kk) & 1;
        cudaStream_t s = (cudaStream_t)stream;
        h->dim = coarse->dim;
        h->family = family;
        h->k = k;
        h->restart = o.restart;
        sfem::Mesh cm;
        cm.d = coarse->dim;
        cm.nv = coarse->n_verts;
        cm.nc = coarse->n_cells;
        cm.X.assign(coarse->verts, coarse->verts + (size_t)cm.nv * cm.d);
        cm.C.assign(coarse->cells, coarse->cells + (size_t)cm.nc * (cm.d + 1));
        sfem::HierarchySpec spec;
        spec.family = family;
        spec.k = k;
        spec.n_refine = n_refine;
        spec.barycentric = barycentric_finest != 0;
        spec.device_assembly = !o.host_only;
        spec.coarsest_first = !o.host_only;
        // the coarsest level's host work beside level 0's, on a thread of its
        // own (the callbacks below are serialised by cb_mu)
        spec.coarsest_thread = !o.host_only;
        spec.device_transfers = !o.host_only && !fbf_mode;
        // (building level 0 before the coarsest level on one thread was
        // slower: with the level-0 inversion already filling the GPU, the
        // coarse factorisation's chain of launches took 5.7 ms and ended
        // after level 0's lambda_max; started first it ends well before)
        if (o.hierarchy == STOKES_HIER_DIRECT) spec.schedule = k > 2 ? std::vector<int>{k, 2} : std::vector<int>{2};
        else if (o.hierarchy == STOKES_HIER_GRADUAL) {
            if (k <= 5) spec.schedule = k > 2 ? std::vector<int>{k, 2} : std::vector<int>{2};
            else if (k <= 7) spec.schedule = {k, 4, 2};
            else spec.schedule = {k, 5, 2};
        } else if (o.hierarchy == STOKES_HIER_EXPLICIT) {
            require(o.n_schedule >= 1 && o.n_schedule <= 8 && o.schedule[0] == k, "explicit schedule must start at k");
            spec.schedule.assign(o.schedule, o.schedule + o.n_schedule);
            for (size_t i = 1; i < spec.schedule.size(); ++i)
                require(spec.schedule[i] >= 2 && spec.schedule[i] < spec.schedule[i - 1], "schedule must decrease");
        } else if (o.hierarchy == STOKES_HIER_HMG) {
            spec.schedule = {k};
        } else {
            require(false, "unknown hierarchy");
        }
        require(fbf_mode || !(family == STOKES_SV && spec.schedule.size() < 2),
                "Scott-Vogelius needs at least one p-coarsening");
        const bool want32 = o.precision == STOKES_MIXED;
        double t_cb_upload = 0;
        std::unique_ptr<Launcher> launcher;
        double t_launch = 0;
        std::function<void(int, int)> on_level;
        std::mutex cb_mu;                  // the callbacks come from two host threads
        if (!o.host_only) {
            // level-by-level pipeline: upload on s_up, then the patch
            // inversion (or the coarse factorisation) starts on the device
            // while the host assembles the next, coarser levels
            // uploads get the highest stream priority: pageable copies on this
            // node run through the SMs, and must not queue behind the patch
            // inversion that occupies every SM
            int prio_lo = 0, prio_hi = 0;
            CK(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
            // (a greater priority is a numerically smaller value)
            auto prio = [&](int steps_below_top) { return std::min(prio_lo, prio_hi + steps_below_top); };
            CK(cudaStreamCreateWithPriority(&h->s_up, cudaStreamNonBlocking, prio(0)));
            // level 0 (the critical path: largest inversion, then its
            // lambda_max estimate) runs on its own stream one step below the
            // uploads; the other relaxed levels one step lower, each on its
            // own stream so that their inversions and lambda_max estimates
            // overlap each other and level 0's.  The coarse factorisation is
            // a chain of dependent launches whose own SM time is small: top
            // priority, so that its CTAs (a 16-CTA cluster per panel) are
            // placed ahead of the patch inversions' waiting CTAs
            CK(cudaStreamCreateWithPriority(&h->s_coarse, cudaStreamNonBlocking, prio(0)));
            CK(cudaStreamCreateWithPriority(&h->s_tr, cudaStreamNonBlocking, prio(3)));
            const int prio_l0 = prio(1), prio_small = prio(2);
            {
                // level 0's stream starts after whatever the caller queued on s
                h->s_lvl.assign(1, nullptr);
                CK(cudaStreamCreateWithPriority(&h->s_lvl[0], cudaStreamNonBlocking, prio_l0));
                cudaEvent_t ev;
                CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
                CK(cudaEventRecord(ev, s));
                CK(cudaStreamWaitEvent(h->s_lvl[0], ev, 0));
                CK(cudaEventDestroy(ev));
            }
            launcher.reset(new Launcher());
            // order the launcher's work on `target` after everything queued on s_up so far
            auto after_uploads = [](stokes_mg* hp, cudaStream_t target) {
                cudaEvent_t ev;
                CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
                CK(cudaEventRecord(ev, hp->s_up));
                CK(cudaStreamWaitEvent(target, ev, 0));
                CK(cudaEventDestroy(ev));
            };
            // device transfers: after the uploads on s_up, on their own stream
            auto launch_transfer = [&](std::function<void()> job) {
                after_uploads(h.get(), h->s_tr);
                stokes_mg* hp0 = h.get();
                launcher->submit([hp0, job] {
                    CK(cudaSetDevice(hp0->device));
                    job();
                });
            };
            on_level = [&](int li, int stage) {
                std::lock_guard<std::mutex> cb_guard(cb_mu);
                const double tu = host_ms();
                stokes_mg* hp = h.get();
                CK(cudaSetDevice(hp->device));    // the callback may run on a helper thread
                const int nlv = (int)hp->H.levels.size();
                if ((int)hp->L.size() != nlv) {
                    hp->L.assign(nlv, DevLevel());
                    hp->kws.resize(nlv);      // sized once: launches keep pointers into it
                    alloc_hess(hp, hp->s_up);
                    hp->s_lvl.resize(nlv, nullptr);
                    for (int x = 1; x + 1 < nlv; ++x)
                        CK(cudaStreamCreateWithPriority(&hp->s_lvl[x], cudaStreamNonBlocking, prio_small));
                }
                // uploads on this thread; relaxed level l then computes on
                // s_lvl[l], the coarse level on s_coarse
                const bool relaxed = li + 1 < nlv;
                cudaStream_t target = relaxed ? hp->s_lvl[li] : hp->s_coarse;
                if (stage == 0) {
                    // operator: the device assembly starts while the host
                    // builds the patches
                    if (!relaxed) return;
                    upload_level_operator(hp, li, want32, hp->s_up);
                    mark(hp, "L" + std::to_string(li) + " operator uploaded", hp->s_up);
                    after_uploads(hp, target);
                    t_cb_upload += host_ms() - tu;
                    launcher->submit([hp, li, target] {
                        CK(cudaSetDevice(hp->device));
                        mark(hp, "L" + std::to_string(li) + " device start", target);
                        assemble_on_device(hp, li, target);
                        mark(hp, "L" + std::to_string(li) + " assembled", target);
                    });
                    if (spec.device_transfers) {
                        // P_{l-1} once level l's maps are up (levels are
                        // built finest to coarsest); P_l too when the next
                        // level is the coarsest and its maps are up already
                        hp->L[li].maps_up = true;
                        if (li >= 1) build_transfer_dev(hp, li - 1, want32, launch_transfer);
                        if (li + 2 == nlv && hp->L[li + 1].maps_up) build_transfer_dev(hp, li, want32, launch_transfer);
                    }
                    return;
                }
                if (relaxed) {
                    upload_level_patches(hp, li, want32, hp->s_up);
                    const double tk = host_ms();
                    if (li == 0) alloc_krylov(hp, hp->s_up);
                    else alloc_level_krylov(hp, li, hp->s_up);
                    trace("krylov buffers", li, tk);
                } else {
                    upload_level_operator(hp, li, want32, hp->s_up);
                    upload_coarse(hp, hp->s_up);
                    if (spec.device_transfers) {
                        // the coarse side of the last transfer
                        const sfem::Level& HC = hp->H.levels[li];
                        hp->L[li].am.vcell = hupload(hp, HC.V.cell_nodes, hp->s_up);
                        hp->L[li].am.qcell = hupload(hp, HC.Q.cell_nodes, hp->s_up);
                        hp->L[li].am.vfree = hupload(hp, HC.vfree, hp->s_up);
                        hp->L[li].maps_up = true;
                        // the last transfer now if its fine level came first
                        if (nlv >= 2 && hp->L[nlv - 2].maps_up && !hp->L[nlv - 2].dev_transfer)
                            build_transfer_dev(hp, nlv - 2, want32, launch_transfer);
                    }
                }
                mark(hp, "L" + std::to_string(li) + " uploaded", hp->s_up);
                after_uploads(hp, target);
                t_cb_upload += host_ms() - tu;
                trace("level callback total", li, tu);
                // kernel launches on the launcher thread
                launcher->submit([hp, li, nlv, target, &o, &t_launch] {
                    const double tl = host_ms();
                    CK(cudaSetDevice(hp->device));
                    if (li + 1 < nlv) {
                        const cudaStream_t sl = target;
                        launch_patches(hp, li, sl);
                        mark(hp, "L" + std::to_string(li) + " inverted", sl);
                        // lambda_max estimate right behind the inversion (same stream)
                        if (!(li < 16 && o.lmax_override[li] > 0)) {
                            const int n = hp->L[li].n;
                            const KrylovWS* ws = li == 0 ? nullptr : &hp->kws[li];
                            double* v0 = li == 0 ? hp->v0buf : ws->v0;
                            splitmix_uniform<<<grid_for(n), 256, 0, sl>>>(n, o.eig_seed, (unsigned long long)li, v0);
                            CK(cudaGetLastError());
                            const size_t hsz = (size_t)skern::HESS_MAX * skern::HESS_MAX;
                            hp->arn_m[li] = arnoldi_launch(hp, li, v0, o.eig_steps, hp->Hlev + li * hsz,
                                                           hp->pinned_H + (li + 1) * hsz, sl, ws);
                            mark(hp, "L" + std::to_string(li) + " arnoldi", sl);
                        }
                    } else {
                        mark(hp, "coarse start", hp->s_coarse);
                        launch_coarse(hp, hp->s_coarse);
                        mark(hp, "coarse factorised", hp->s_coarse);
                    }
                    t_launch += host_ms() - tl;
                });
            };
        }
        if (fbf_mode) {
            // FBF(phMG): the SV Stokes hierarchy is built on the host for its
            // operators only; the handle's levels become its scalar velocity
            // hierarchy (ASMStarPC patches), set up level by level as below
            sfem::HierarchySpec sp = spec;
            sp.device_assembly = !o.host_only;
            sp.device_assembly_finest_only = true;
            sp.coarsest_first = false;
            sp.skip_patches = true;
            sp.device_transfers = false;       // the velocity hierarchy takes blocks of the host transfers
            sfem::Hierarchy S;
            sfem::build_hierarchy(cm, sp, nu_cell, S, nullptr);
            h->fbf.reset(new FbfData());
            FbfData& F = *h->fbf;
            sfem::velocity_hierarchy(S, h->H);
            F.S0 = std::move(S.levels[0]);
            F.nS = F.S0.n_free;
            F.nvf = F.S0.nVf;
            F.nu = F.S0.d * F.S0.nVf;
            h->H.t_mesh_ms = S.t_mesh_ms;
            h->H.t_assembly_ms = S.t_assembly_ms;
            h->H.t_spaces_ms = S.t_spaces_ms;
            h->H.t_matrices_ms = S.t_matrices_ms;
            h->H.t_transfers_ms = S.t_transfers_ms;
            h->opts.patch_solver = 1;          // dense SPD star blocks: Gauss-Jordan
            const int nlv = (int)h->H.levels.size();
            if (on_level) {
                on_level(nlv - 1, 0);
                on_level(nlv - 1, 1);
                // level 0: the device-assembled Stokes K and its velocity block
                stokes_mg* hp = h.get();
                const cudaStream_t s0 = hp->s_lvl[0];
                fbf_level0_operator(hp, want32, s0);
                launcher->submit([hp, s0] {
                    CK(cudaSetDevice(hp->device));
                    fbf_level0_kernels(hp, s0);
                });
                on_level(0, 1);
                for (int li = 1; li + 1 < nlv; ++li) {
                    on_level(li, 0);
                    on_level(li, 1);
                }
            }
        } else {
            sfem::build_hierarchy(cm, spec, nu_cell, h->H, on_level);
        }
        if (!o.host_only) {
            mark(h.get(), "host hierarchy built", h->s_up);
            alloc_readback(h.get());
        }
        h->st.t_mesh_ms = h->H.t_mesh_ms;
        h->st.t_assembly_ms = h->H.t_assembly_ms;
        h->st.t_spaces_ms = h->H.t_spaces_ms;
        h->st.t_matrices_ms = h->H.t_matrices_ms;
        h->st.t_patches_ms = h->H.t_patches_ms;
        h->st.t_transfers_ms = h->H.t_transfers_ms;
        const int nl = (int)h->H.levels.size();
        require(nl >= 2, "the hierarchy needs at least two levels (n_refine >= 1 or a p-coarsening)");
        if (o.host_only) {
            h->host_only = true;
            h->st.t_total_ms = host_ms() - t0;
            fill_stats(h.get());
            return STOKES_OK;
        }
        double t1 = host_ms();
        launcher->finish();   // all per-level uploads and launches issued
        const double t_wait_launch = host_ms() - t1;
        t1 = host_ms();
        for (int li = 0; li + 1 < nl; ++li) upload_transfers(h.get(), li, want32, h->s_up);
        const int n0 = h->L[0].n;
        setup_solve_buffers(h.get(), h->s_up);
        if (h->fbf) setup_fbf(h.get(), h->s_up);
        mark(h.get(), "transfers uploaded", h->s_up);
        CK(cudaStreamSynchronize(h->s_up));
        h->st.t_upload_ms = t_cb_upload;
        h->st.t_upload_post_ms = host_ms() - t1;
        h->st.t_launch_wait_ms = t_wait_launch;
        h->st.t_launch_thread_ms = t_launch;
        // what remains of the patch inversions, the lambda_max estimates and
        // the coarse factorisation once the host is done (one wait)
        t1 = host_ms();
        finish_setup(h.get(), s);
        h->st.t_gather_lu_ms = host_ms() - t1;
        h->st.t_coarse_ms = 0;
        t1 = host_ms();
        {
            const size_t hsz = (size_t)skern::HESS_MAX * skern::HESS_MAX;
            for (int li = 0; li + 1 < nl; ++li) {
                if (li < 16 && o.lmax_override[li] > 0) { h->L[li].lmax = o.lmax_override[li]; continue; }
                h->L[li].lmax = arnoldi_finish(h->pinned_H + (li + 1) * hsz, h->arn_m[li]);
                if (!(h->L[li].lmax > 0) || !std::isfinite(h->L[li].lmax))
                    throw StokesError(STOKES_ENONFINITE, "lambda_max estimate is not positive on level " + std::to_string(li));
            }
        }
        h->st.t_eig_ms = host_ms() - t1;
        t1 = host_ms();
        if (o.use_graph) capture_graph(h.get(), o.precision, s);
        h->st.t_graph_ms = host_ms() - t1;
        h->st.t_total_ms = host_ms() - t0;
        mark(h.get(), "setup end", s);
        print_marks(h.get());
        fill_stats(h.get());
        return STOKES_OK;
    });
    if (rc != STOKES_OK) {
        stokes_mg_destroy(h.release());
        return rc;
    }
    *out = h.release();
    return STOKES_OK;
}
}  // namespace

int stokes_mg_setup(const stokes_mesh* coarse, int n_refine, int barycentric_finest, int family, int k,
                    const stokes_mg_opts* opts, const double* nu_cell, void* stream, stokes_mg_t* out) {
    return setup_impl(coarse, n_refine, barycentric_finest, family, k, opts, nu_cell, stream, out, false);
}

int stokes_fbf_setup(const stokes_mesh* coarse, int n_refine, int k, const stokes_mg_opts* opts, const double* nu_cell,
                     void* stream, stokes_mg_t* out) {
    return setup_impl(coarse, n_refine, 1, STOKES_SV, k, opts, nu_cell, stream, out, true);
}

int stokes_fbf_apply(stokes_mg_t h, const double* r_dev, double* z_dev, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && r_dev && z_dev, "invalid argument");
        require(h->fbf != nullptr, "not an FBF handle (stokes_fbf_setup)");
        DeviceGuard dg(h);
        fbf_apply(h, r_dev, z_dev, (cudaStream_t)stream);
        return STOKES_OK;
    });
}

int stokes_mg_vcycle(stokes_mg_t h, const double* r_dev, double* z_dev, int nrhs, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && r_dev && z_dev && nrhs >= 1, "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        const int n = h->L[0].n;
        for (int q = 0; q < nrhs; ++q) {
            CK(cudaMemcpyAsync(h->vin, r_dev + (size_t)q * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            vcycle_run(h, h->opts.precision, s);
            CK(cudaMemcpyAsync(z_dev + (size_t)q * n, h->vout, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        }
        return STOKES_OK;
    });
}

namespace {
// batched V-cycle of an interleaved FP64 batch (width h->bm): Z = B_MG V
void batched_precond(stokes_mg* h, int mode, const double* V, double* Z, cudaStream_t s) {
    const int m = h->bm;
    ensure_plan(h, mode, m, s);
    const long long nm = (long long)h->L[0].n * m;
    launch(h, -1, s, [&] { sbat::to32(nm, V, h->bl[0].b, s); });
    const bool any_prof = h->prof[PK_PATCH].on || h->prof[PK_SPMV].on || h->prof[PK_PULL].on || h->prof[PK_TRANSFER].on;
    if (h->opts.use_graph && !any_prof) {
        if (!h->bgraph[mode]) capture_batched(h, mode, m);
        CK(cudaGraphLaunch(h->bgraph[mode], s));
        h->launches += h->bgraph_launches[mode];
    } else {
        b_pcycle(h, 0, mode, m, h->bl[0].b, h->bl[0].e, s);
    }
    launch(h, -1, s, [&] { sbat::to64(nm, h->bl[0].e, Z, s); });
}

void ensure_bkrylov(stokes_mg* h, int m) {
    auto& K = h->bk;
    if (K.m == m) return;
    const size_t nm = (size_t)h->L[0].n * m;
    const int R = h->restart, ldh = R + 1;
    K.V = halloc<double>(h, (size_t)(R + 1) * nm);
    K.Z = halloc<double>(h, (size_t)R * nm);
    K.W = halloc<double>(h, nm);
    K.R = halloc<double>(h, nm);
    K.B = halloc<double>(h, nm);
    K.X = halloc<double>(h, nm);
    K.partial = halloc<double>(h, sbat::col_partial_doubles(m));
    K.hcol = halloc<double>(h, (size_t)32 * m);
    K.hcol2 = halloc<double>(h, (size_t)32 * m);
    K.hn = halloc<double>(h, m);
    K.Hc = halloc<double>(h, (size_t)m * ldh * ldh);
    K.cs = halloc<double>(h, (size_t)m * ldh);
    K.sn = halloc<double>(h, (size_t)m * ldh);
    K.g = halloc<double>(h, (size_t)m * (ldh + 1));
    K.y = halloc<double>(h, (size_t)m * (ldh + 1));
    K.resid = halloc<double>(h, m);
    K.beta = halloc<double>(h, m);
    K.beta0 = halloc<double>(h, m);
    if (!K.host) CK(cudaMallocHost((void**)&K.host, sizeof(double) * 2 * 64));
    CK(cudaStreamSynchronize(h->s_up));
    K.m = m;
}

// nrhs independent FGMRES(restart) solves (Sec. 4) in lockstep, every
// column right-preconditioned by the batched V-cycle; x0 = 0, column c
// stops counting once ||b_c - K x_c|| <= tol ||b_c|| (estimate), the batch
// once every column has.  Krylov arithmetic in FP64, CGS2 as the
// single-vector solver, deterministic.
int fgmres_batched(stokes_mg* h, int nrhs, int mode, const double* B_dev, double* X_dev, double tol, int* its_out,
                   double* rel_out, cudaStream_t s) {
    const int m = nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : nrhs <= 32 ? 32 : 64;
    ensure_batch(h, m);
    ensure_bkrylov(h, m);
    auto& K = h->bk;
    DevLevel& l0 = h->L[0];
    const int n = l0.n, R = h->restart, ldh = R + 1;
    const long long nm = (long long)n * m;
    launch(h, -1, s, [&] { sbat::pack64(n, nrhs, m, B_dev, K.B, s); });
    CK(cudaMemsetAsync(K.X, 0, sizeof(double) * nm, s));
    launch(h, -1, s, [&] { sbat::col_dots(n, m, 1, K.B, 0, K.B, K.partial, K.beta0, 1, 0, s); });
    CK(cudaMemcpyAsync(K.host, K.beta0, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> beta0(K.host, K.host + m), res(m, 0.0);
    for (int c = 0; c < nrhs; ++c)
        if (!std::isfinite(beta0[c])) throw StokesError(STOKES_ENONFINITE, "non-finite right-hand side");
    auto all_done = [&](const std::vector<double>& r) {
        for (int c = 0; c < nrhs; ++c)
            if (beta0[c] > 0.0 && !(r[c] <= tol * beta0[c])) return false;
        return true;
    };
    CK(cudaMemcpyAsync(K.R, K.B, sizeof(double) * nm, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(K.beta, K.beta0, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    int its = 0;
    bool converged = all_done(beta0);      // only zero right-hand sides
    while (!converged && its < h->opts.maxit) {
        launch(h, -1, s, [&] { sbat::col_start(m, ldh + 1, K.beta, K.g, s); });
        launch(h, -1, s, [&] { sbat::col_scale(n, m, K.R, K.beta, K.V, s); });
        int jend = 0;
        for (int j = 0; j < R; ++j) {
            const double* Vj = K.V + (long long)j * nm;
            double* Zj = K.Z + (long long)j * nm;
            batched_precond(h, mode, Vj, Zj, s);
            launch(h, PK_SPMV, s, [&] { sbat::spmm64(0, n, m, l0.K.rp, l0.K.ci, l0.K.v64, Zj, K.W, nullptr, s); });
            // CGS2
            launch(h, -1, s, [&] { sbat::col_dots(n, m, j + 1, K.V, nm, K.W, K.partial, K.hcol, 0, 0, s); });
            launch(h, -1, s, [&] { sbat::col_update(n, m, j + 1, K.V, nm, K.hcol, K.W, s); });
            launch(h, -1, s, [&] { sbat::col_dots(n, m, j + 1, K.V, nm, K.W, K.partial, K.hcol2, 0, 0, s); });
            launch(h, -1, s, [&] { sbat::col_update(n, m, j + 1, K.V, nm, K.hcol2, K.W, s); });
            axpby_l<double>(h, (j + 1) * m, 1.0, K.hcol2, 1.0, K.hcol, s);
            launch(h, -1, s, [&] { sbat::col_dots(n, m, 1, K.W, 0, K.W, K.partial, K.hn, 1, 0, s); });
            launch(h, -1, s, [&] { sbat::col_scale(n, m, K.W, K.hn, K.V + (long long)(j + 1) * nm, s); });
            launch(h, -1, s, [&] { sbat::col_givens(j, m, ldh, K.Hc, K.hcol, K.hn, K.cs, K.sn, K.g, K.resid, s); });
            CK(cudaMemcpyAsync(K.host, K.resid, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            res.assign(K.host, K.host + m);
            for (int c = 0; c < nrhs; ++c)
                if (!std::isfinite(res[c])) throw StokesError(STOKES_ENONFINITE, "non-finite FGMRES residual");
            ++its;
            jend = j + 1;
            if (all_done(res)) { converged = true; break; }
            if (its >= h->opts.maxit) break;
        }
        launch(h, -1, s, [&] { sbat::col_backsolve(jend, m, ldh, K.Hc, K.g, K.y, s); });
        launch(h, -1, s, [&] { sbat::col_xupdate(n, m, jend, ldh + 1, K.Z, nm, K.y, K.X, s); });
        if (converged) break;
        // restart: the true residual of every column
        launch(h, PK_SPMV, s, [&] { sbat::spmm64(2, n, m, l0.K.rp, l0.K.ci, l0.K.v64, K.X, K.R, K.B, s); });
        launch(h, -1, s, [&] { sbat::col_dots(n, m, 1, K.R, 0, K.R, K.partial, K.beta, 1, 0, s); });
        CK(cudaMemcpyAsync(K.host, K.beta, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        res.assign(K.host, K.host + m);
        if (all_done(res)) converged = true;
    }
    launch(h, -1, s, [&] { sbat::unpack64(n, nrhs, m, K.X, X_dev, s); });
    if (its_out) *its_out = its;
    if (rel_out)
        for (int c = 0; c < nrhs; ++c) rel_out[c] = beta0[c] > 0.0 ? res[c] / beta0[c] : 0.0;
    return converged ? STOKES_OK : STOKES_ENOTCONVERGED;
}

// b = stokes_solve's free-DoF right-hand side for the nodal forcing f and
// Dirichlet data g (NULL: homogeneous): b_u = (M f)/nu - K[free, D] g on the
// free velocity rows, b_p = -K[p, D] g, then the pressure part made
// orthogonal to the constant pressures (the consistency condition of the
// singular all-Dirichlet system, Sec. 2)
void solve_rhs(stokes_mg* h, const double* f_nodal, const double* g_nodal, double nu, double* b, cudaStream_t s) {
    const sfem::Level& F = finest_stokes(h);
    const int d = F.d, nV = F.V.n, nVf = F.nVf, nQ = F.nQ;
    const double* gfull = g_nodal ? g_nodal : h->gzero;
    const DevLevel& fl = h->fbf ? h->fbf->S0d : h->L[0];
    if (fl.dev_asm) {
        // matrix-free: assembled per row from the incident cells (the same
        // element integrals as the operator)
        launch(h, -1, s, [&] { sasm::load_vector(fl.am, f_nodal, g_nodal, 1.0 / nu, b, s); });
    } else {
        // F_c = M f_c
        for (int c = 0; c < d; ++c)
            spmv<double>(h, -1, h->Mv, skern::SPMV_SET, f_nodal + (size_t)c * nV, h->F + (size_t)c * nV, nullptr, s);
        launch(h, -1, s, [&] { skern::gather_idx<double><<<grid_for(d * nVf), 256, 0, s>>>(d * nVf, h->vel_rows, h->F, b); });
        if (nu != 1.0) axpby_l<double>(h, d * nVf, 0.0, b, 1.0 / nu, b, s);
        CK(cudaMemsetAsync(b + (size_t)d * nVf, 0, sizeof(double) * nQ, s));
        spmv<double>(h, -1, h->KfD, skern::SPMV_RESID, gfull, b, b, s);
    }
    mdot(h, nQ, 1, b + (size_t)d * nVf, nQ, h->ones, h->scal, nullptr, false, s);
    launch(h, -1, s, [&] { skern::sub_scalar<<<grid_for(nQ), 256, 0, s>>>(nQ, b + (size_t)d * nVf, h->scal, (double)nQ); });
}

// (u, p) from the free-DoF solution x: u = g on the boundary and x on the
// free nodes; p = nu * p' shifted to int p = 0 (Sec. 2)
void solve_output(stokes_mg* h, const double* x, const double* g_nodal, double nu, double* u, double* p,
                  cudaStream_t s) {
    const sfem::Level& F = finest_stokes(h);
    const int d = F.d, nV = F.V.n, nVf = F.nVf, nQ = F.nQ;
    const double* gfull = g_nodal ? g_nodal : h->gzero;
    CK(cudaMemcpyAsync(u, gfull, sizeof(double) * d * nV, cudaMemcpyDeviceToDevice, s));
    launch(h, -1, s, [&] { skern::scatter_idx<double><<<grid_for(d * nVf), 256, 0, s>>>(d * nVf, h->vel_rows, x, u); });
    CK(cudaMemcpyAsync(p, x + (size_t)d * nVf, sizeof(double) * nQ, cudaMemcpyDeviceToDevice, s));
    if (nu != 1.0) axpby_l<double>(h, nQ, 0.0, p, nu, p, s);
    mdot(h, nQ, 1, p, nQ, h->pint, h->scal, nullptr, false, s);
    launch(h, -1, s, [&] { skern::sub_scalar<<<grid_for(nQ), 256, 0, s>>>(nQ, p, h->scal, h->pint_sum); });
}

// r = (gu on the free velocity DoFs, nu Pi^T gp), Pi^T gp = gp - w (1^T gp) / (w^T 1):
// the transpose of the zero-mean normalisation of the solve's pressure output
void adjoint_rhs(stokes_mg* h, const double* gu, const double* gp, double nu, double* r, cudaStream_t s) {
    const sfem::Level& F = finest_stokes(h);
    const int d = F.d, nVf = F.nVf, nQ = F.nQ;
    double* rp = r + (size_t)d * nVf;
    launch(h, -1, s, [&] { skern::gather_idx<double><<<grid_for(d * nVf), 256, 0, s>>>(d * nVf, h->vel_rows, gu, r); });
    CK(cudaMemcpyAsync(rp, gp, sizeof(double) * nQ, cudaMemcpyDeviceToDevice, s));
    mdot(h, nQ, 1, rp, nQ, h->ones, h->scal, nullptr, false, s);
    launch(h, -1, s, [&] { skern::sub_weighted<<<grid_for(nQ), 256, 0, s>>>(nQ, rp, h->pint, h->scal, h->pint_sum); });
    if (nu != 1.0) axpby_l<double>(h, nQ, 0.0, rp, nu, rp, s);
}

// lambda_u (0 on the boundary), lambda_p (zero plain mean; optional) and
// dL/df_c = M lambda_u,c / nu (optional) from the free-DoF adjoint x
void adjoint_output(stokes_mg* h, const double* x, double nu, double* lam_u, double* lam_p, double* grad_f,
                    cudaStream_t s) {
    const sfem::Level& F = finest_stokes(h);
    const int d = F.d, nV = F.V.n, nVf = F.nVf, nQ = F.nQ;
    CK(cudaMemsetAsync(lam_u, 0, sizeof(double) * d * nV, s));
    launch(h, -1, s, [&] { skern::scatter_idx<double><<<grid_for(d * nVf), 256, 0, s>>>(d * nVf, h->vel_rows, x, lam_u); });
    if (lam_p) {
        CK(cudaMemcpyAsync(lam_p, x + (size_t)d * nVf, sizeof(double) * nQ, cudaMemcpyDeviceToDevice, s));
        mdot(h, nQ, 1, lam_p, nQ, h->ones, h->scal, nullptr, false, s);
        launch(h, -1, s, [&] { skern::sub_scalar<<<grid_for(nQ), 256, 0, s>>>(nQ, lam_p, h->scal, (double)nQ); });
    }
    if (grad_f) {
        const DevLevel& fl = h->fbf ? h->fbf->S0d : h->L[0];
        if (fl.dev_asm) {
            launch(h, -1, s, [&] { sasm::mass_apply_all(fl.am, lam_u, 1.0 / nu, grad_f, s); });
        } else {
            for (int c = 0; c < d; ++c)
                spmv<double>(h, -1, h->Mv, skern::SPMV_SET, lam_u + (size_t)c * nV, grad_f + (size_t)c * nV, nullptr, s);
            if (nu != 1.0) axpby_l<double>(h, d * nV, 0.0, grad_f, 1.0 / nu, grad_f, s);
        }
    }
}

// argument checks shared by the batched entries: a monolithic MIXED handle
// whose patches all fit the batched patch GEMM at this width
void require_batched(stokes_mg* h, int nrhs, int mode) {
    require(nrhs >= 1 && nrhs <= STOKES_BATCH_MAX, "nrhs must be in 1..STOKES_BATCH_MAX");
    require(mode == STOKES_BATCH_TF32 || mode == STOKES_BATCH_3XTF32, "unknown batch mode");
    require(!h->host_only && h->opts.precision == STOKES_MIXED && !h->fbf,
            "the batched FGMRES needs a monolithic MIXED handle");
    require(h->L[0].K.v64 != nullptr, "level 0 has no FP64 operator");
    const int m = nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : nrhs <= 32 ? 32 : 64;
    for (size_t li = 0; li + 1 < h->L.size(); ++li)
        if (const char* why = sbat::patch_gemm_check(mode, h->L[li].maxn, m))
            throw StokesError(STOKES_EUNSUPPORTED, why);
}

// the batched solve entries' free-DoF right-hand sides and solutions,
// [width][n_free(level 0)] each, kept for the handle's lifetime
void ensure_batch_io(stokes_mg* h, int nrhs) {
    auto& K = h->bk;
    const int m = nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : nrhs <= 32 ? 32 : 64;
    if (K.io_m >= m) return;
    const size_t nm = (size_t)h->L[0].n * m;
    K.iob = halloc<double>(h, nm);
    K.iox = halloc<double>(h, nm);
    CK(cudaStreamSynchronize(h->s_up));
    K.io_m = m;
}
}  // namespace

int stokes_selftest_bounded_wait(long long polls, int* result) {
    g_last_error.clear();
    return guarded([&] {
        require(result && polls >= 0, "invalid argument");
        int* d = nullptr;
        CK(cudaMalloc((void**)&d, sizeof(int)));
        CK(cudaMemset(d, 0, sizeof(int)));
        const int e = sbat::wait_probe(polls, d, nullptr);
        if (e != cudaSuccess) { cudaFree(d); CK((cudaError_t)e); }
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(result, d, sizeof(int), cudaMemcpyDeviceToHost));
        CK(cudaFree(d));
        return STOKES_OK;
    });
}

int stokes_probe_fp64_peak(long long iters, int blocks_per_sm, double* tflops, float* ms, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(tflops && ms && iters >= 1 && blocks_per_sm >= 1 && blocks_per_sm <= 8, "invalid argument");
        int dev = 0, nsm = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const cudaStream_t s = (cudaStream_t)stream;
        const int grid = nsm * blocks_per_sm;
        double* out = nullptr;
        CK(cudaMallocAsync((void**)&out, sizeof(double) * grid, s));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        // warm-up launch, then the timed one
        skern::fp64_fma_probe<<<grid, 256, 0, s>>>(iters / 8 + 1, 0.999999, 1e-7, -1.0, out);
        CK(cudaEventRecord(e0, s));
        skern::fp64_fma_probe<<<grid, 256, 0, s>>>(iters, 0.999999, 1e-7, -1.0, out);
        CK(cudaEventRecord(e1, s));
        CK(cudaGetLastError());
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        CK(cudaEventDestroy(e0));
        CK(cudaEventDestroy(e1));
        CK(cudaFreeAsync(out, s));
        CK(cudaStreamSynchronize(s));
        *tflops = 2.0 * 8.0 * (double)iters * 256.0 * grid / (*ms * 1e-3) / 1e12;
        return STOKES_OK;
    });
}

int stokes_fgmres_batched(stokes_mg_t h, const double* b_dev, double* x_dev, int nrhs, int mode, double tol,
                          int* iterations, double* final_relres, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && b_dev && x_dev && tol > 0, "invalid argument");
        require_batched(h, nrhs, mode);
        DeviceGuard dg(h);
        int rc = fgmres_batched(h, nrhs, mode, b_dev, x_dev, tol, iterations, final_relres, (cudaStream_t)stream);
        if (rc != STOKES_OK) g_last_error = "batched FGMRES: a column did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_batch_plan(stokes_mg_t h, int mode, int level, int max_parts, int* n_parts, int* kind, int* warps,
                      int* count, int* lo, int* hi, double* part_us, double* single_us) {
    g_last_error.clear();
    return guarded([&] {
        require(h && n_parts && (mode == STOKES_BATCH_TF32 || mode == STOKES_BATCH_3XTF32), "invalid argument");
        require(level >= 0 && level + 1 < (int)h->L.size() && level < (int)h->bl.size(), "no such relaxed level");
        const auto& plan = h->bl[level].plan[mode];
        require(!plan.empty(), "no batched call in this mode at the current width yet");
        *n_parts = (int)plan.size();
        for (int i = 0; i < (int)plan.size() && i < max_parts; ++i) {
            if (kind) kind[i] = plan[i].kind;
            if (warps) warps[i] = plan[i].nw;
            if (count) count[i] = plan[i].count;
            if (lo) lo[i] = plan[i].lo;
            if (hi) hi[i] = plan[i].hi;
            if (part_us) part_us[i] = plan[i].us;
        }
        if (single_us) *single_us = h->bl[level].single_us[mode];
        return STOKES_OK;
    });
}

int stokes_mg_vcycle_batched(stokes_mg_t h, const double* r_dev, double* z_dev, int nrhs, int mode, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && r_dev && z_dev && nrhs >= 1 && nrhs <= STOKES_BATCH_MAX, "invalid argument");
        require(mode == STOKES_BATCH_TF32 || mode == STOKES_BATCH_3XTF32, "unknown batch mode");
        require(!h->host_only && h->opts.precision == STOKES_MIXED,
                "the batched V-cycle needs a MIXED handle (FP32 operators and inverses)");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        const int m = nrhs <= 8 ? 8 : nrhs <= 16 ? 16 : nrhs <= 32 ? 32 : 64;
        for (size_t li = 0; li + 1 < h->L.size(); ++li)
            if (const char* why = sbat::patch_gemm_check(mode, h->L[li].maxn, m))
                throw StokesError(STOKES_EUNSUPPORTED, why);
        if (h->bstat_h && *(volatile int*)h->bstat_h) {
            *(volatile int*)h->bstat_h = 0;
            throw StokesError(STOKES_ECUDA, "a tensor-core patch GEMM of an earlier batched V-cycle timed out on "
                                            "its mbarrier; its output was not written");
        }
        ensure_batch(h, m);
        ensure_plan(h, mode, m, s);
        const int n = h->L[0].n;
        launch(h, -1, s, [&] { sbat::to_interleaved(n, nrhs, m, r_dev, h->bl[0].b, s); });
        const bool any_prof = h->prof[PK_PATCH].on || h->prof[PK_SPMV].on || h->prof[PK_PULL].on ||
                              h->prof[PK_TRANSFER].on;
        if (h->opts.use_graph && !any_prof) {
            if (!h->bgraph[mode]) capture_batched(h, mode, m);
            CK(cudaGraphLaunch(h->bgraph[mode], s));
            h->launches += h->bgraph_launches[mode];
        } else {
            b_pcycle(h, 0, mode, m, h->bl[0].b, h->bl[0].e, s);
        }
        launch(h, -1, s, [&] { sbat::from_interleaved(n, nrhs, m, h->bl[0].e, z_dev, s); });
        return STOKES_OK;
    });
}

int stokes_mg_fgmres(stokes_mg_t h, const double* b, double* x, double tol, int* iterations, double* final_relres,
                     void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && b && x && tol > 0, "invalid argument");
        DeviceGuard dg(h);
        int rc = fgmres(h, b, x, tol, iterations, final_relres, (cudaStream_t)stream);
        if (rc != STOKES_OK) g_last_error = "FGMRES did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_solve(stokes_mg_t h, const double* f_nodal, const double* g_nodal, double nu, double tol, double* u,
                 double* p, int* iterations, double* final_relres, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && f_nodal && u && p, "invalid argument");
        require(nu > 0 && std::isfinite(nu) && tol > 0, "nu and tol must be positive");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        solve_rhs(h, f_nodal, g_nodal, nu, h->bvec, s);
        int rc = fgmres(h, h->bvec, h->xvec, tol, iterations, final_relres, s);
        solve_output(h, h->xvec, g_nodal, nu, u, p, s);
        if (rc != STOKES_OK) g_last_error = "FGMRES did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_adjoint_solve(stokes_mg_t h, const double* gu, const double* gp, double nu, double tol, double* lam_u,
                         double* lam_p, double* grad_f, int* iterations, double* final_relres, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && gu && gp && lam_u, "invalid argument");
        require(nu > 0 && std::isfinite(nu) && tol > 0, "nu and tol must be positive");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        adjoint_rhs(h, gu, gp, nu, h->bvec, s);
        // K is symmetric: the adjoint system is the forward one (same FGMRES-phMG)
        int rc = fgmres(h, h->bvec, h->xvec, tol, iterations, final_relres, s);
        adjoint_output(h, h->xvec, nu, lam_u, lam_p, grad_f, s);
        if (rc != STOKES_OK) g_last_error = "FGMRES did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_grad_viscosity(stokes_mg_t h, const double* u, const double* lam_u, double* grad, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && u && lam_u && grad, "invalid argument");
        DeviceGuard dg(h);
        const DevLevel& fl = h->fbf ? h->fbf->S0d : h->L[0];
        if (!fl.dev_asm)
            throw StokesError(STOKES_EUNSUPPORTED, "the viscosity gradient needs a device-assembled finest level");
        cudaStream_t s = (cudaStream_t)stream;
        launch(h, -1, s, [&] { sasm::grad_viscosity(fl.am, u, lam_u, 1, 0, grad, s); });
        return STOKES_OK;
    });
}

int stokes_grad_viscosity_batched(stokes_mg_t h, const double* u, const double* lam_u, int nrhs, double* grad,
                                  void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && u && lam_u && grad && nrhs >= 1, "invalid argument");
        DeviceGuard dg(h);
        const DevLevel& fl = h->fbf ? h->fbf->S0d : h->L[0];
        if (!fl.dev_asm)
            throw StokesError(STOKES_EUNSUPPORTED, "the viscosity gradient needs a device-assembled finest level");
        const sfem::Level& F = finest_stokes(h);
        const long long ld = (long long)F.d * F.V.n;
        cudaStream_t s = (cudaStream_t)stream;
        launch(h, -1, s, [&] { sasm::grad_viscosity(fl.am, u, lam_u, nrhs, ld, grad, s); });
        return STOKES_OK;
    });
}

int stokes_solve_batched(stokes_mg_t h, const double* f_nodal, const double* g_nodal, int nrhs, int mode, double nu,
                         double tol, double* u, double* p, int* iterations, double* final_relres, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && f_nodal && u && p, "invalid argument");
        require(nu > 0 && std::isfinite(nu) && tol > 0, "nu and tol must be positive");
        require_batched(h, nrhs, mode);
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        ensure_batch_io(h, nrhs);
        const sfem::Level& F = finest_stokes(h);
        const long long nv = (long long)F.d * F.V.n, n = F.n_free, nQ = F.nQ;
        auto& K = h->bk;
        for (int q = 0; q < nrhs; ++q)
            solve_rhs(h, f_nodal + q * nv, g_nodal ? g_nodal + q * nv : nullptr, nu, K.iob + q * n, s);
        int rc = fgmres_batched(h, nrhs, mode, K.iob, K.iox, tol, iterations, final_relres, s);
        for (int q = 0; q < nrhs; ++q)
            solve_output(h, K.iox + q * n, g_nodal ? g_nodal + q * nv : nullptr, nu, u + q * nv, p + q * nQ, s);
        if (rc != STOKES_OK) g_last_error = "batched FGMRES: a column did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_adjoint_solve_batched(stokes_mg_t h, const double* gu, const double* gp, int nrhs, int mode, double nu,
                                 double tol, double* lam_u, double* lam_p, double* grad_f, int* iterations,
                                 double* final_relres, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && gu && gp && lam_u, "invalid argument");
        require(nu > 0 && std::isfinite(nu) && tol > 0, "nu and tol must be positive");
        require_batched(h, nrhs, mode);
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        ensure_batch_io(h, nrhs);
        const sfem::Level& F = finest_stokes(h);
        const long long nv = (long long)F.d * F.V.n, n = F.n_free, nQ = F.nQ;
        auto& K = h->bk;
        for (int q = 0; q < nrhs; ++q) adjoint_rhs(h, gu + q * nv, gp + q * nQ, nu, K.iob + q * n, s);
        int rc = fgmres_batched(h, nrhs, mode, K.iob, K.iox, tol, iterations, final_relres, s);
        for (int q = 0; q < nrhs; ++q)
            adjoint_output(h, K.iox + q * n, nu, lam_u + q * nv, lam_p ? lam_p + q * nQ : nullptr,
                           grad_f ? grad_f + q * nv : nullptr, s);
        if (rc != STOKES_OK) g_last_error = "batched FGMRES: a column did not reach the tolerance within maxit";
        return rc;
    });
}

int stokes_mg_cell_centroids(stokes_mg_t h, int* n_cells, double* xyz) {
    g_last_error.clear();
    return guarded([&] {
        require(h && n_cells, "invalid argument");
        const sfem::Mesh& m = h->H.meshes[0];
        *n_cells = m.nc;
        if (xyz)
            for (int e = 0; e < m.nc; ++e)
                for (int c = 0; c < m.d; ++c) {
                    double x = 0;
                    for (int v = 0; v <= m.d; ++v) x += m.X[(size_t)m.C[(size_t)e * (m.d + 1) + v] * m.d + c];
                    xyz[(size_t)e * m.d + c] = x / (m.d + 1);
                }
        return STOKES_OK;
    });
}

int stokes_mg_info(stokes_mg_t h, stokes_mg_stats* st) {
    if (!h || !st) { g_last_error = "invalid argument"; return STOKES_EINVAL; }
    fill_stats(h);
    h->st.kernel_launches = h->launches;
    *st = h->st;
    return STOKES_OK;
}

int stokes_mg_level_dofs(stokes_mg_t h, int level, double* xyz, int* comp, double* cell_center) {
    g_last_error.clear();
    return guarded([&] {
        require(h && level >= 0 && level < (int)h->H.levels.size() && xyz && comp, "invalid argument");
        const sfem::Level& L = h->H.levels[level];
        const int d = L.d;
        std::vector<int> vrow(L.nVf);
        for (int i = 0; i < L.V.n; ++i)
            if (L.vfree[i] >= 0) vrow[L.vfree[i]] = i;
        for (int r = 0; r < L.n_free; ++r) {
            const double* x;
            if (r < d * L.nVf) {
                comp[r] = r / L.nVf;
                x = &L.V.X[(size_t)vrow[r % L.nVf] * d];
            } else {
                comp[r] = d;
                x = &L.Q.X[(size_t)(r - d * L.nVf) * d];
            }
            for (int c = 0; c < d; ++c) xyz[(size_t)r * d + c] = x[c];
            if (cell_center) {
                for (int c = 0; c < d; ++c) cell_center[(size_t)r * d + c] = 0.0;
                if (r >= d * L.nVf && !L.Q.continuous) {
                    const int e = L.Q.owner_cell[r - d * L.nVf];
                    for (int c = 0; c < d; ++c) cell_center[(size_t)r * d + c] = L.cell_center[(size_t)e * d + c];
                }
            }
        }
        return STOKES_OK;
    });
}

int stokes_mg_nodes(stokes_mg_t h, double* vel_xyz, double* pres_xyz, double* pres_cell_center) {
    g_last_error.clear();
    return guarded([&] {
        require(h, "invalid argument");
        const sfem::Level& L = finest_stokes(h);
        const int d = L.d;
        if (vel_xyz) std::memcpy(vel_xyz, L.V.X.data(), sizeof(double) * L.V.X.size());
        if (pres_xyz) std::memcpy(pres_xyz, L.Q.X.data(), sizeof(double) * L.Q.X.size());
        if (pres_cell_center)
            for (int q = 0; q < L.nQ; ++q)
                for (int c = 0; c < d; ++c)
                    pres_cell_center[(size_t)q * d + c] = L.Q.continuous ? 0.0 : L.cell_center[(size_t)L.Q.owner_cell[q] * d + c];
        return STOKES_OK;
    });
}

int stokes_mg_get_csr(stokes_mg_t h, int level, int which, int* n_rows, int* n_cols, long long* nnz, int* row_ptr,
                      int* col, double* val) {
    g_last_error.clear();
    return guarded([&] {
        const int nl = h ? (int)h->H.levels.size() : 0;
        require(h && level >= 0 && level < nl && which >= 0 && which <= 2, "invalid argument");
        const sfem::Level& L = h->H.levels[level];
        require(which == 0 || level + 1 < nl, "no transfer on the coarsest level");
        if (which == 0 && !L.host_matrices) {
            // assembled on the device
            const DevCSR& D = h->L[level].K;
            if (n_rows) *n_rows = D.nr;
            if (n_cols) *n_cols = D.nc;
            if (nnz) *nnz = D.nnz;
            if (row_ptr) {
                CK(cudaMemcpy(row_ptr, D.rp, sizeof(int) * (D.nr + 1), cudaMemcpyDeviceToHost));
                if (col) CK(cudaMemcpy(col, D.ci, sizeof(int) * D.nnz, cudaMemcpyDeviceToHost));
                if (val) CK(cudaMemcpy(val, D.v64, sizeof(double) * D.nnz, cudaMemcpyDeviceToHost));
            }
            return STOKES_OK;
        }
        if (which != 0 && level < (int)h->L.size() && h->L[level].dev_transfer) {
            // built on the device
            const DevCSR& D = which == 1 ? h->L[level].P : h->L[level].R;
            if (n_rows) *n_rows = D.nr;
            if (n_cols) *n_cols = D.nc;
            if (nnz) *nnz = D.nnz;
            if (row_ptr) {
                CK(cudaMemcpy(row_ptr, D.rp, sizeof(int) * (D.nr + 1), cudaMemcpyDeviceToHost));
                if (col) CK(cudaMemcpy(col, D.ci, sizeof(int) * D.nnz, cudaMemcpyDeviceToHost));
                if (val) CK(cudaMemcpy(val, D.v64, sizeof(double) * D.nnz, cudaMemcpyDeviceToHost));
            }
            return STOKES_OK;
        }
        const sfem::CSR& A = which == 0 ? L.K : (which == 1 ? L.P : L.R);
        if (n_rows) *n_rows = A.nr;
        if (n_cols) *n_cols = A.ncol;
        if (nnz) *nnz = A.nnz();
        if (row_ptr) {
            std::memcpy(row_ptr, A.rp.data(), sizeof(int) * (A.nr + 1));
            if (col) std::memcpy(col, A.ci.data(), sizeof(int) * A.nnz());
            if (val) std::memcpy(val, A.v.data(), sizeof(double) * A.nnz());
        }
        return STOKES_OK;
    });
}

int stokes_mg_get_patches(stokes_mg_t h, int level, int* n_patches, long long* n_entries, int* offsets, int* dofs) {
    g_last_error.clear();
    return guarded([&] {
        require(h && level >= 0 && level + 1 < (int)h->H.levels.size(), "invalid argument");
        const sfem::Level& HL = h->H.levels[level];
        if (n_patches) *n_patches = (int)HL.patch_off.size() - 1;
        if (n_entries) *n_entries = (long long)HL.patch_dofs.size();
        if (offsets) std::memcpy(offsets, HL.patch_off.data(), sizeof(int) * HL.patch_off.size());
        if (dofs) std::memcpy(dofs, HL.patch_dofs.data(), sizeof(int) * HL.patch_dofs.size());
        return STOKES_OK;
    });
}

int stokes_mg_patch_matrices(stokes_mg_t h, int level, double* out, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && out && level >= 0 && level + 1 < (int)h->L.size(), "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel& l = h->L[level];
        double* work = dalloc<double>(l.nsq);
        launch(h, -1, s, [&] { skern::fill_vec<double><<<grid_for(l.nsq), 256, 0, s>>>(l.nsq, 0.0, work); });
        launch(h, -1, s, [&] {
            skern::patch_gather<<<l.npatch, 256, l.maxn * sizeof(int), s>>>(l.npatch, l.poff, l.pdofs, l.moff, l.K.rp,
                                                                           l.K.ci, l.K.v64, work);
        });
        cudaError_t e = cudaMemcpyAsync(out, work, sizeof(double) * l.nsq, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(work);
        CK(e);
        return STOKES_OK;
    });
}

int stokes_mg_patch_inverses(stokes_mg_t h, int level, double* out, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && out && level >= 0 && level + 1 < (int)h->L.size(), "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel& l = h->L[level];
        double* work = dalloc<double>(l.nsq);
        int* status = dalloc<int>(l.npatch);
        cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int) * l.npatch, s);
        try {
            gather_and_invert(h, level, work, INV_BACK, status, s);
        } catch (...) {
            cudaFree(work);
            cudaFree(status);
            throw;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, work, sizeof(double) * l.nsq, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(work);
        cudaFree(status);
        CK(e);
        return STOKES_OK;
    });
}

int stokes_mg_arnoldi_lmax(stokes_mg_t h, int level, const double* v0_dev, int steps, double* lmax, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && v0_dev && lmax && level >= 0 && level + 1 < (int)h->L.size() && steps >= 1 && steps <= 15,
                "invalid argument");
        DeviceGuard dg(h);
        *lmax = arnoldi_lmax(h, level, v0_dev, steps, (cudaStream_t)stream);
        return STOKES_OK;
    });
}

int stokes_mg_residual(stokes_mg_t h, int level, const double* b, const double* x, double* r, int precision,
                       void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && b && x && r && level >= 0 && level < (int)h->L.size(), "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel& l = h->L[level];
        if (precision == STOKES_FP64) {
            spmv<double>(h, PK_SPMV, l.K, skern::SPMV_RESID, x, r, b, s);
        } else {
            require(l.K.v32, "mixed precision needs a MIXED handle");
            Tmp32 tb(l.n), tx(l.n), tr(l.n);
            skern::convert_vec<float, double><<<grid_for(l.n), 256, 0, s>>>(l.n, b, tb.p);
            skern::convert_vec<float, double><<<grid_for(l.n), 256, 0, s>>>(l.n, x, tx.p);
            spmv<float>(h, PK_SPMV, l.K, skern::SPMV_RESID, tx.p, tr.p, tb.p, s);
            skern::convert_vec<double, float><<<grid_for(l.n), 256, 0, s>>>(l.n, tr.p, r);
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaGetLastError());
        return STOKES_OK;
    });
}

int stokes_mg_asm(stokes_mg_t h, int level, const double* r, double* z, int precision, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && r && z && level >= 0 && level + 1 < (int)h->L.size(), "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel& l = h->L[level];
        if (precision == STOKES_FP64) {
            asm_apply<double>(h, l, r, z, 1.0, 0.0, s);
        } else {
            require(l.inv32 || l.fac32, "mixed precision needs a MIXED handle");
            Tmp32 tr(l.n), tz(l.n);
            skern::convert_vec<float, double><<<grid_for(l.n), 256, 0, s>>>(l.n, r, tr.p);
            asm_apply<float>(h, l, tr.p, tz.p, 1.0, 0.0, s);
            skern::convert_vec<double, float><<<grid_for(l.n), 256, 0, s>>>(l.n, tz.p, z);
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaGetLastError());
        return STOKES_OK;
    });
}

int stokes_mg_transfer(stokes_mg_t h, int level, int dir, const double* x, double* y, int precision, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && x && y && level >= 0 && level + 1 < (int)h->L.size() && (dir == 0 || dir == 1), "invalid argument");
        DeviceGuard dg(h);
        cudaStream_t s = (cudaStream_t)stream;
        DevLevel& l = h->L[level];
        const DevCSR& A = dir == 0 ? l.R : l.P;
        const int mode = dir == 0 ? skern::SPMV_SET : skern::SPMV_ADD;
        if (precision == STOKES_FP64) {
            spmv<double>(h, PK_TRANSFER, A, mode, x, y, nullptr, s);
        } else {
            require(A.v32, "mixed precision needs a MIXED handle");
            Tmp32 tx(A.nc), ty(A.nr);
            skern::convert_vec<float, double><<<grid_for(A.nc), 256, 0, s>>>(A.nc, x, tx.p);
            skern::convert_vec<float, double><<<grid_for(A.nr), 256, 0, s>>>(A.nr, y, ty.p);
            spmv<float>(h, PK_TRANSFER, A, mode, tx.p, ty.p, nullptr, s);
            skern::convert_vec<double, float><<<grid_for(A.nr), 256, 0, s>>>(A.nr, ty.p, y);
            CK(cudaStreamSynchronize(s));
        }
        CK(cudaGetLastError());
        return STOKES_OK;
    });
}

int stokes_mg_coarse_solve(stokes_mg_t h, const double* r, double* x, void* stream) {
    g_last_error.clear();
    return guarded([&] {
        require(h && r && x, "invalid argument");
        DeviceGuard dg(h);
        coarse_apply<double>(h, r, x, (cudaStream_t)stream);
        return STOKES_OK;
    });
}

int stokes_prof_enable(stokes_mg_t h, int kind, int enable) {
    if (!h || kind < 0 || kind >= 5) { g_last_error = "invalid argument"; return STOKES_EINVAL; }
    h->prof[kind].on = enable != 0;
    return STOKES_OK;
}

static void prof_resolve(Prof& p) {
    for (auto& ab : p.pending) {
        CK(cudaEventSynchronize(ab.second));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, ab.first, ab.second));
        p.total_ms += ms;
        p.each_ms.push_back(ms);
        cudaEventDestroy(ab.first);
        cudaEventDestroy(ab.second);
    }
    p.pending.clear();
}

int stokes_prof_read(stokes_mg_t h, int kind, long long* launches, double* total_ms) {
    g_last_error.clear();
    return guarded([&] {
        require(h && kind >= 0 && kind < 5, "invalid argument");
        Prof& p = h->prof[kind];
        prof_resolve(p);
        if (launches) *launches = p.launches;
        if (total_ms) *total_ms = p.total_ms;
        return STOKES_OK;
    });
}

int stokes_prof_read_one(stokes_mg_t h, int kind, long long index, double* ms) {
    g_last_error.clear();
    return guarded([&] {
        require(h && kind >= 0 && kind < 5 && ms, "invalid argument");
        Prof& p = h->prof[kind];
        prof_resolve(p);
        require(index >= 0 && index < (long long)p.each_ms.size(), "launch index out of range");
        *ms = p.each_ms[index];
        return STOKES_OK;
    });
}

void stokes_mg_destroy(stokes_mg_t h) {
    if (!h) return;
    if (h->host_only || (h->allocs.empty() && !h->pinned)) { delete h; return; }
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != h->device) cudaSetDevice(h->device);
    for (auto& p : h->prof)
        for (auto& ab : p.pending) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
    if (h->s_up || h->s_coarse) cudaDeviceSynchronize();
    for (auto* m : h->marks) delete m;
    for (int i = 0; i < 2; ++i) {
        if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
        if (h->bgraph[i]) cudaGraphExecDestroy(h->bgraph[i]);
    }
    if (h->s_up || h->s_coarse) cudaDeviceSynchronize();   // setup work may still be in flight after an error
    free_pending(h);
    free_coarse_ws(h);
    if (h->s_up) cudaStreamDestroy(h->s_up);
    for (cudaStream_t x : h->s_lvl)
        if (x) cudaStreamDestroy(x);
    if (h->s_coarse) cudaStreamDestroy(h->s_coarse);
    if (h->s_tr) cudaStreamDestroy(h->s_tr);
    for (void* p : h->allocs) cudaFree(p);
    if (!h->pool_allocs.empty()) {
        for (void* p : h->pool_allocs) cudaFreeAsync(p, 0);
        cudaStreamSynchronize(0);
    }
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->pinned_rb) cudaFreeHost(h->pinned_rb);
    if (h->pinned_H) cudaFreeHost(h->pinned_H);
    if (h->bstat_h) cudaFreeHost(h->bstat_h);
    if (h->bk.host) cudaFreeHost(h->bk.host);
    if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
    delete h;
}

}  // extern "C"
