// stokes_batched_inverse_noalloc: the batched FP64 Gauss-Jordan patch
// inversion for callers that cannot allocate device memory.
//
// Who needs it: an application whose device memory is owned by another
// allocator (a framework's caching pool that has already reserved the HBM,
// so cudaMalloc fails or fragments it), or code that must never enter the
// CUDA allocator at all (cudaFree synchronises the whole device).  Such a
// caller owns the matrices it passes in and receives the inverses in place;
// every other buffer the kernels need (patch offsets, pivot status, and the
// pivot / column workspace of patches too large for shared memory) lives in
// a file-scope __device__ array of fixed size, g_noalloc_scratch below.
// Every GPU that loads this library holds that array until the process
// exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/stokes_mg.h"
#include "kernels.cuh"

namespace {

constexpr int kMaxPatches = STOKES_NOALLOC_MAX_PATCHES;
constexpr long long kMaxEntries = STOKES_NOALLOC_MAX_ENTRIES;
constexpr int kMaxDevices = 64;

// scratch layout (each part 256-byte aligned):
//   poff   int       [kMaxPatches + 1]   patch offsets (sum of sizes)
//   moff   long long [kMaxPatches + 1]   matrix offsets (sum of size^2)
//   status int       [kMaxPatches]       0 or 1 + step of the first zero pivot
//   ipiv   int       [kMaxEntries]       pivot rows (patches > shared-memory limit)
//   col    double    [kMaxEntries]       pivot column copies (same)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffPoff = 0;
constexpr size_t kOffMoff = align256(kOffPoff + sizeof(int) * (kMaxPatches + 1));
constexpr size_t kOffStatus = align256(kOffMoff + sizeof(long long) * (kMaxPatches + 1));
constexpr size_t kOffIpiv = align256(kOffStatus + sizeof(int) * kMaxPatches);
constexpr size_t kOffCol = align256(kOffIpiv + sizeof(int) * kMaxEntries);
constexpr size_t kScratchBytes = align256(kOffCol + sizeof(double) * kMaxEntries);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host copies of the offsets and of the status array (static, not allocated),
// shared by every thread of the process.  g_call_mu serialises whole calls:
// a call holds it from filling these arrays until its stream has drained and
// the status has been read back, so concurrent host calls (on one device or
// on several) never overwrite each other's offsets or status.  std::mutex
// has a constexpr constructor and locks through the kernel's futex: no heap.
static int h_poff[kMaxPatches + 1];
static long long h_moff[kMaxPatches + 1];
static int h_status[kMaxPatches];
static std::mutex g_call_mu;

// Device address of g_noalloc_scratch, looked up once per device: in host
// code the symbol's name is only a host-side stand-in and must never be
// handed to a kernel.
static unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};

// error text in a fixed buffer: this entry point allocates nothing, not even
// on the host
thread_local char g_err[160];

int fail(int code, const char* msg, long long arg = -1) {
    if (arg >= 0) std::snprintf(g_err, sizeof(g_err), "%s %lld", msg, arg);
    else std::snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

}  // namespace

extern "C" const char* stokes_noalloc_last_error(void) { return g_err; }

extern "C" int stokes_batched_inverse_noalloc(int npatch, const int* sizes, double* mats, int* first_singular,
                                              void* stream) {
    g_err[0] = 0;
    if (first_singular) *first_singular = -1;
    if (npatch < 1 || npatch > kMaxPatches || !sizes || !mats)
        return fail(STOKES_EINVAL, "npatch must be in [1, STOKES_NOALLOC_MAX_PATCHES] and pointers non-NULL");
    std::lock_guard<std::mutex> call_lock(g_call_mu);
    long long total = 0;
    int nmax = 0;
    h_poff[0] = 0;
    h_moff[0] = 0;
    for (int p = 0; p < npatch; ++p) {
        const int n = sizes[p];
        if (n < 1 || n > 4096) return fail(STOKES_EINVAL, "patch size must be in [1, 4096]");
        total += n;
        if (total > kMaxEntries)
            return fail(STOKES_EINVAL, "sum of patch sizes exceeds STOKES_NOALLOC_MAX_ENTRIES");
        nmax = n > nmax ? n : nmax;
        h_poff[p + 1] = (int)total;
        h_moff[p + 1] = h_moff[p] + (long long)n * n;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(STOKES_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(STOKES_EUNSUPPORTED, "device index beyond the supported range");
    if (!g_scratch_addr[dev]) {
        // set-up on the first call on this device, with that device current
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) return fail(STOKES_ECUDA, cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char*)ptr;
    }
    unsigned char* base = g_scratch_addr[dev];
    int* poff = (int*)(base + kOffPoff);
    long long* moff = (long long*)(base + kOffMoff);
    int* status = (int*)(base + kOffStatus);
    int* ipiv = (int*)(base + kOffIpiv);
    double* col = (double*)(base + kOffCol);
    cudaStream_t s = (cudaStream_t)stream;
    // the offsets come from pageable static host memory: the copies are
    // staged before cudaMemcpyAsync returns, so the next call may refill them
    if ((e = cudaMemcpyAsync(poff, h_poff, sizeof(int) * (npatch + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(moff, h_moff, sizeof(long long) * (npatch + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(status, 0, sizeof(int) * npatch, s)) != cudaSuccess)   // every call starts from zero status
        return fail(STOKES_ECUDA, cudaGetErrorString(e));
    const int nsm = nmax < skern::GJ_SMEM_MAX_N ? nmax : skern::GJ_SMEM_MAX_N;
    const size_t smem = (size_t)nsm * nsm * sizeof(double) + nsm * sizeof(double) + nsm * sizeof(int) + 64;
    // The attribute is process-wide and the setup path launches the same
    // kernel from other threads and streams: always set the one upper bound
    // (the largest shared-memory patch) that the setup path sets, never a
    // smaller value, and launch with this call's own smaller size.
    {
        const size_t gmax = skern::GJ_SMEM_MAX_N;
        const size_t smem_max = gmax * gmax * sizeof(double) + gmax * sizeof(double) + gmax * sizeof(int) + 64;
        if ((e = cudaFuncSetAttribute(skern::gj_inverse_smem, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_max)) != cudaSuccess)
            return fail(STOKES_ECUDA, cudaGetErrorString(e));
    }
    skern::gj_inverse_smem<<<npatch, 256, smem, s>>>(npatch, poff, moff, mats, nullptr, nullptr, nullptr, nullptr, status, 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(STOKES_ECUDA, cudaGetErrorString(e));
    if (nmax > skern::GJ_SMEM_MAX_N) {
        skern::gj_inverse_global<<<npatch, 512, 0, s>>>(npatch, poff, moff, mats, nullptr, nullptr, nullptr, nullptr,
                                                        status, ipiv, col);
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(STOKES_ECUDA, cudaGetErrorString(e));
    }
    if ((e = cudaMemcpyAsync(h_status, status, sizeof(int) * npatch, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(STOKES_ECUDA, cudaGetErrorString(e));
    for (int p = 0; p < npatch; ++p)
        if (h_status[p] != 0) {
            if (first_singular) *first_singular = p;
            return fail(STOKES_ESINGULAR, "zero pivot in patch", p);
        }
    return STOKES_OK;
}
