// Host-side finite-element setup; see fem.hpp.
#include "fem.hpp"

#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <numeric>
#include <stdexcept>
#include <exception>
#include <thread>
#include <unordered_map>
#include <unordered_set>

namespace sfem {

int num_threads() {
    static int n = [] {
        const char* e = std::getenv("STOKES_HOST_THREADS");
        int v = e ? std::atoi(e) : (int)std::thread::hardware_concurrency();
        return std::max(1, std::min(v, 64));
    }();
    return n;
}

// CSR row pointers, column indices and list offsets are 32-bit: a total
// beyond that range is rejected (std::length_error) before any array is sized
static int index_total(long long n, const char* what) {
    if (n > INT32_MAX)
        throw std::length_error(std::string(what) + " beyond 2^31 - 1 entries (32-bit indices)");
    return (int)n;
}

// set on a thread that must not use the shared pool (the coarsest level's
// builder): its parallel loops run inline
thread_local bool t_pool_inline = false;

// Persistent worker pool: parallel_for splits [0, n) into one contiguous,
// ordered chunk per worker (the caller runs chunk 0).  A job is published
// under the mutex with a new generation; workers that spin on the
// generation (bounded, yielding, then asleep on the condition variable)
// register for it under the mutex, so they read its fields consistently, and
// claim chunks with an atomic counter.  The caller retires the job under the
// mutex once every chunk is done and waits for the registered workers to
// leave it, so no worker touches a finished job.  (The wake through the
// condition variable alone cost tens of microseconds per parallel loop.)
class Pool {
  public:
    static Pool& get() {
        static Pool p(num_threads());
        return p;
    }
    int size() const { return (int)workers_.size() + 1; }
    void run(int chunks, const std::function<void(int)>& job) {
        if (chunks <= 1 || workers_.empty() || t_pool_inline) {
            for (int c = 0; c < chunks; ++c) job(c);
            return;
        }
        std::lock_guard<std::mutex> serial(run_mu_);     // one job at a time
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = &job;
            chunks_ = chunks;
            next_.store(1, std::memory_order_relaxed);
            done_.store(0, std::memory_order_relaxed);
            gen_.fetch_add(1, std::memory_order_release);
        }
        if (sleepers_.load(std::memory_order_acquire) > 0) cv_.notify_all();
        run_chunk(job, 0);
        for (int c; (c = next_.fetch_add(1, std::memory_order_acq_rel)) < chunks;) run_chunk(job, c);
        while (done_.load(std::memory_order_acquire) < chunks) std::this_thread::yield();
        std::exception_ptr err;
        {
            std::lock_guard<std::mutex> lk(m_);
            job_ = nullptr;
            err = err_;
            err_ = nullptr;
        }
        while (active_.load(std::memory_order_acquire) > 0) std::this_thread::yield();
        if (err) std::rethrow_exception(err);
    }
    ~Pool() {
        {
            std::lock_guard<std::mutex> lk(m_);
            stop_.store(true, std::memory_order_release);
            gen_.fetch_add(1, std::memory_order_release);
        }
        cv_.notify_all();
        for (auto& t : workers_) t.join();
    }

  private:
    explicit Pool(int n) {
        for (int i = 1; i < n; ++i) workers_.emplace_back([this] { loop(); });
    }
    // one chunk; its exception (the first) is kept for the caller, and the
    // chunk still counts as done so that the job completes.  A parallel loop
    // nested inside a chunk runs inline (the pool runs one job at a time).
    void run_chunk(const std::function<void(int)>& job, int c) {
        const bool was_inline = t_pool_inline;
        t_pool_inline = true;
        try {
            job(c);
        } catch (...) {
            std::lock_guard<std::mutex> lk(m_);
            if (!err_) err_ = std::current_exception();
        }
        t_pool_inline = was_inline;
        done_.fetch_add(1, std::memory_order_acq_rel);
    }
    void loop() {
        unsigned seen = 0;
        for (;;) {
            // wait for a new generation: spin (yielding) for about kSpinUs,
            // then sleep on the condition variable
            auto t0 = std::chrono::steady_clock::now();
            for (int spin = 0; gen_.load(std::memory_order_acquire) == seen; ++spin) {
                if (stop_.load(std::memory_order_acquire)) return;
                if ((spin & 63) != 63 ||
                    std::chrono::steady_clock::now() - t0 < std::chrono::microseconds(kSpinUs)) {
                    std::this_thread::yield();
                    continue;
                }
                std::unique_lock<std::mutex> lk(m_);
                sleepers_.fetch_add(1, std::memory_order_acq_rel);
                cv_.wait(lk, [&] {
                    return gen_.load(std::memory_order_acquire) != seen || stop_.load(std::memory_order_acquire);
                });
                sleepers_.fetch_sub(1, std::memory_order_acq_rel);
                spin = 0;
                t0 = std::chrono::steady_clock::now();
            }
            const std::function<void(int)>* j = nullptr;
            int ch = 0;
            {
                std::lock_guard<std::mutex> lk(m_);
                if (stop_.load(std::memory_order_acquire)) return;
                seen = gen_.load(std::memory_order_acquire);
                if (!job_) continue;                         // already retired
                j = job_;
                ch = chunks_;
                active_.fetch_add(1, std::memory_order_acq_rel);
            }
            for (int c; (c = next_.fetch_add(1, std::memory_order_acq_rel)) < ch;) run_chunk(*j, c);
            active_.fetch_sub(1, std::memory_order_acq_rel);
        }
    }
    static constexpr int kSpinUs = 300;                       // spin before sleeping
    std::vector<std::thread> workers_;
    std::mutex m_, run_mu_;
    std::condition_variable cv_;
    const std::function<void(int)>* job_ = nullptr;          // guarded by m_
    std::exception_ptr err_;                                  // guarded by m_
    int chunks_ = 0;                                          // guarded by m_
    std::atomic<int> next_{0}, done_{0}, active_{0}, sleepers_{0};
    std::atomic<unsigned> gen_{0};
    std::atomic<bool> stop_{false};
};

// chunks for n items of at least `grain` items each (1 = run inline: waking
// the workers costs more than a light loop over a few thousand items)
static int chunk_count(int n, int grain = 64) { return std::max(1, std::min(Pool::get().size(), n / grain)); }

// Parallel loop over [0, n) in contiguous chunks of at least `grain` items:
// body(lo, hi, chunk), chunk < Pool::size() unless split > 1 (then up to
// split chunks per thread, claimed as threads come free, so that a thread
// that is descheduled holds back less of the loop).
static void parallel_for(int n, const std::function<void(int, int, int)>& body, int grain = 64, int split = 1) {
    const int T = std::max(1, std::min(Pool::get().size() * std::max(1, split), n / grain));
    Pool::get().run(T, [&](int t) {
        int lo = (int)((long long)n * t / T), hi = (int)((long long)n * (t + 1) / T);
        body(lo, hi, t);
    });
}

void parallel_copy(void* dst, const void* src, size_t bytes) {
    const size_t chunk = 1 << 20;
    const int n = (int)((bytes + chunk - 1) / chunk);
    const int T = std::max(1, std::min(Pool::get().size(), n));
    Pool::get().run(T, [&](int t) {
        const size_t lo = bytes * t / T, hi = bytes * (t + 1) / T;
        std::memcpy((char*)dst + lo, (const char*)src + lo, hi - lo);
    });
}

// Variable-length lists built in parallel without per-item allocations:
// the static chunks of parallel_for are contiguous and ordered, so the
// per-thread buffers concatenate in item order.
struct FlatLists {
    std::vector<int> off;
    fvec<int> data;
    const int* begin(int i) const { return data.data() + off[i]; }
    int size(int i) const { return off[i + 1] - off[i]; }
};

// fill(i, out, t) appends item i's list to out; t is the chunk, below
// Pool::size() unless split > 1 (then up to split chunks per thread, claimed
// as threads come free: a thread that is descheduled holds back less work)
template <class F>
static FlatLists build_lists(int n, F&& fill, int per_item = 32, int split = 1) {
    const int T = std::max(1, std::min(Pool::get().size() * std::max(1, split), n / 64));
    std::vector<std::vector<int>> buf(T);
    FlatLists L;
    L.off.assign(n + 1, 0);
    std::vector<int> lo(T + 1);
    for (int t = 0; t <= T; ++t) lo[t] = (int)((long long)n * t / T);
    Pool::get().run(T, [&](int t) {
        std::vector<int>& b = buf[t];
        b.reserve((size_t)(lo[t + 1] - lo[t]) * per_item);
        for (int i = lo[t]; i < lo[t + 1]; ++i) {
            size_t before = b.size();
            fill(i, b, t);
            L.off[i + 1] = (int)(b.size() - before);
        }
    });
    long long total = 0;
    for (int i = 0; i < n; ++i) {
        total += L.off[i + 1];
        L.off[i + 1] = index_total(total, "index lists");
    }
    L.data.resize(L.off[n]);
    parallel_for(T, [&](int a, int b2, int) {
        for (int t = a; t < b2; ++t)
            if (!buf[t].empty()) std::memcpy(L.data.data() + L.off[lo[t]], buf[t].data(), buf[t].size() * sizeof(int));
    });
    return L;
}

// Sort out[s0..) and drop repeated values, in place.  A list whose values
// span a narrow range (a vertex star: its nodes are numbered close together)
// is marked in a bit map of that range, which is then read back in order;
// a list over a wide range is sorted.  The bit map is per thread and all
// zero between calls.
static void sort_unique_tail(std::vector<int>& out, size_t s0) {
    thread_local std::vector<uint64_t> bits;
    const size_t n = out.size() - s0;
    if (n <= 1) return;
    int lo = out[s0], hi = out[s0];
    for (size_t i = s0 + 1; i < out.size(); ++i) {
        lo = std::min(lo, out[i]);
        hi = std::max(hi, out[i]);
    }
    const long long words = (((long long)hi - lo) >> 6) + 1;
    if (words > 8 * (long long)n + 64) {
        std::sort(out.begin() + s0, out.end());
        out.erase(std::unique(out.begin() + s0, out.end()), out.end());
        return;
    }
    if ((long long)bits.size() < words) bits.resize((size_t)words, 0);
    for (size_t i = s0; i < out.size(); ++i) {
        const unsigned r = (unsigned)(out[i] - lo);
        bits[r >> 6] |= 1ull << (r & 63);
    }
    size_t w = s0;
    for (long long k = 0; k < words; ++k) {
        uint64_t b = bits[k];
        bits[k] = 0;
        while (b) {
            out[w++] = lo + (int)(k << 6) + __builtin_ctzll(b);
            b &= b - 1;
        }
    }
    out.resize(w);
}

// Parallel exclusive scan of cnt[0..n) into out[0..n] (out[n] = total).
static void parallel_scan(const int* cnt, int n, int* out) {
    const int T = chunk_count(n, 16384);
    std::vector<long long> part(T + 1, 0);
    Pool::get().run(T, [&](int t) {
        const int lo = (int)((long long)n * t / T), hi = (int)((long long)n * (t + 1) / T);
        long long s = 0;
        for (int i = lo; i < hi; ++i) s += cnt[i];
        part[t + 1] = s;
    });
    for (int t = 0; t < T; ++t) part[t + 1] += part[t];
    Pool::get().run(T, [&](int t) {
        const int lo = (int)((long long)n * t / T), hi = (int)((long long)n * (t + 1) / T);
        long long s = part[t];
        for (int i = lo; i < hi; ++i) { out[i] = (int)s; s += cnt[i]; }
    });
    out[n] = (int)part[T];
}

void invert_index(const int* idx, long long m, int n, std::vector<int>& off, std::vector<int>& pos) {
    off.assign(n + 1, 0);
    std::vector<int> cnt(n, 0);
    const int T = (int)std::max<long long>(1, std::min<long long>(Pool::get().size(), m / 8192));
    Pool::get().run(T, [&](int t) {
        const long long lo = m * t / T, hi = m * (t + 1) / T;
        for (long long q = lo; q < hi; ++q) __atomic_fetch_add(&cnt[idx[q]], 1, __ATOMIC_RELAXED);
    });
    parallel_scan(cnt.data(), n, off.data());
    pos.resize(m);
    std::vector<int> cur(off.begin(), off.end() - 1);
    Pool::get().run(T, [&](int t) {
        const long long lo = m * t / T, hi = m * (t + 1) / T;
        for (long long q = lo; q < hi; ++q) pos[__atomic_fetch_add(&cur[idx[q]], 1, __ATOMIC_RELAXED)] = (int)q;
    });
    // restore increasing positions within every list (lists are short)
    parallel_for(n, [&](int lo, int hi, int) {
        for (int i = lo; i < hi; ++i) {
            int* a = pos.data() + off[i];
            const int len = off[i + 1] - off[i];
            for (int x = 1; x < len; ++x)
                for (int y = x; y > 0 && a[y - 1] > a[y]; --y) std::swap(a[y - 1], a[y]);
        }
    }, 4096);
}

static double now_ms() {
    return std::chrono::duration<double, std::milli>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

// STOKES_TRACE=1: times of the host build's phases on stderr
static bool host_trace() {
    static const bool on = [] {
        const char* e = std::getenv("STOKES_TRACE");
        return e && e[0] == '1';
    }();
    return on;
}
struct PhaseClock {
    const char* scope;
    double t;
    explicit PhaseClock(const char* s) : scope(s), t(host_trace() ? now_ms() : 0.0) {}
    void lap(const char* what) {
        if (!host_trace()) return;
        const double n = now_ms();
        std::fprintf(stderr, "[sfem]   %-10s %-22s %7.3f ms\n", scope, what, n - t);
        t = n;
    }
};

// ---------------------------------------------------------------- meshes --
static inline uint64_t edge_key(int a, int b) {
    if (a > b) std::swap(a, b);
    return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
}

Mesh refine_uniform(const Mesh& m, std::vector<int>& parent) {
    const int d = m.d, nvpc = d + 1;
    Mesh r;
    r.d = d;
    std::unordered_map<uint64_t, int> mid;
    mid.reserve((size_t)m.nc * 4);
    r.X = m.X;
    int nv = m.nv;
    auto midpoint = [&](int a, int b) {
        uint64_t key = edge_key(a, b);
        auto it = mid.find(key);
        if (it != mid.end()) return it->second;
        for (int c = 0; c < d; ++c) r.X.push_back(0.5 * (m.X[(size_t)a * d + c] + m.X[(size_t)b * d + c]));
        mid.emplace(key, nv);
        return nv++;
    };
    const int nkids = d == 2 ? 4 : 8;
    r.C.reserve((size_t)m.nc * nkids * nvpc);
    parent.assign((size_t)m.nc * nkids, 0);
    for (int e = 0; e < m.nc; ++e) {
        const int* v = &m.C[(size_t)e * nvpc];
        if (d == 2) {
            int m01 = midpoint(v[0], v[1]), m12 = midpoint(v[1], v[2]), m20 = midpoint(v[2], v[0]);
            int kids[4][3] = {{v[0], m01, m20}, {m01, v[1], m12}, {m20, m12, v[2]}, {m12, m20, m01}};
            for (auto& k : kids) r.C.insert(r.C.end(), k, k + 3);
        } else {
            int a = v[0], b = v[1], c = v[2], w = v[3];
            int ab = midpoint(a, b), ac = midpoint(a, c), aw = midpoint(a, w);
            int bc = midpoint(b, c), bw = midpoint(b, w), cw = midpoint(c, w);
            // Bey's regular subdivision: four corner tetrahedra and the inner
            // octahedron cut along the (ac, bw) diagonal.
            int kids[8][4] = {{a, ab, ac, aw}, {ab, b, bc, bw}, {ac, bc, c, cw}, {aw, bw, cw, w},
                              {ab, ac, aw, bw}, {ab, ac, bc, bw}, {ac, aw, bw, cw}, {ac, bc, bw, cw}};
            for (auto& k : kids) r.C.insert(r.C.end(), k, k + 4);
        }
        for (int i = 0; i < nkids; ++i) parent[(size_t)e * nkids + i] = e;
    }
    r.nv = nv;
    r.nc = m.nc * nkids;
    return r;
}

Mesh refine_alfeld(const Mesh& m, std::vector<int>& parent) {
    const int d = m.d, nvpc = d + 1;
    Mesh r;
    r.d = d;
    r.X = m.X;
    r.X.reserve((size_t)(m.nv + m.nc) * d);
    int nv = m.nv;
    parent.assign((size_t)m.nc * nvpc, 0);
    for (int e = 0; e < m.nc; ++e) {
        const int* v = &m.C[(size_t)e * nvpc];
        for (int c = 0; c < d; ++c) {
            double s = 0;
            for (int i = 0; i < nvpc; ++i) s += m.X[(size_t)v[i] * d + c];
            r.X.push_back(s / nvpc);
        }
        int g = nv++;
        for (int i = 0; i < nvpc; ++i) {       // child i: vertex i replaced by the barycenter
            for (int j = 0; j < nvpc; ++j) r.C.push_back(j == i ? g : v[j]);
            parent[(size_t)e * nvpc + i] = e;
        }
    }
    r.nv = nv;
    r.nc = m.nc * nvpc;
    return r;
}

// ------------------------------------------------------ reference element --

static std::vector<double> lagrange_in_bernstein(const RefElement& e);
static std::vector<double> invert_refined(const std::vector<double>& G, int n, int steps);

void RefElement::init(int d_, int k_) {
    d = d_;
    k = k_;
    alpha.clear();
    mono.clear();
    if (d == 2) {
        for (int j = 0; j <= k; ++j)
            for (int i = 0; i <= k - j; ++i) alpha.push_back({k - i - j, i, j, 0});
        for (int t = 0; t <= k; ++t)
            for (int b = 0; b <= t; ++b) mono.push_back({t - b, b, 0});
    } else {
        for (int l = 0; l <= k; ++l)
            for (int j = 0; j <= k - l; ++j)
                for (int i = 0; i <= k - l - j; ++i) alpha.push_back({k - i - j - l, i, j, l});
        for (int t = 0; t <= k; ++t)
            for (int c = 0; c <= t; ++c)
                for (int b = 0; b <= t - c; ++b) mono.push_back({t - b - c, b, c});
    }
    nb = (int)alpha.size();
    nm = (int)mono.size();
    if (nb != nm) throw std::runtime_error("reference element: node/monomial count mismatch");
    // Vandermonde V[node][m] = xi^mono_m with xi = alpha / k.  Scaled by
    // k^|m| per column it is an integer matrix (entries prod alpha^m, at most
    // k^k, exact in double), inverted as given with iterative refinement;
    // then coef[i][m] = k^|m| Vhat^-1[m][i].
    const int n = nb;
    std::vector<double> V((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int m = 0; m < n; ++m) {
            long long v = 1;
            for (int c = 0; c < d; ++c)
                for (int p = 0; p < mono[m][c]; ++p) v *= alpha[i][c + 1];
            V[(size_t)i * n + m] = (double)v;
        }
    const std::vector<double> X = invert_refined(V, n, 4);   // cond up to 2e11 at k = 10 in 3D
    coef.assign((size_t)n * n, 0.0);
    for (int m = 0; m < n; ++m) {
        double scale = 1.0;
        for (int c = 0; c < d; ++c)
            for (int p = 0; p < mono[m][c]; ++p) scale *= k;
        for (int i = 0; i < n; ++i) coef[(size_t)i * n + m] = X[(size_t)m * n + i] * scale;
    }
    bcoef = lagrange_in_bernstein(*this);
}

// Reference tensors through the Bernstein basis.  B_beta = n!/beta! lambda^beta
// (|beta| = n, lambda_0 = 1 - sum xi, lambda_c = xi_c) are nonnegative, and
// the Lagrange basis on the equispaced lattice has moderate coefficients in
// them (below 1.5e3 at k = 10), while its monomial coefficients reach 1e9 and
// their exact integrals cancel to a few digits at high k.  Integrals of
// Bernstein products have a closed form with positive terms:
//   int_T B_beta^m B_gamma^n = m! n! / (beta! gamma!) (beta + gamma)! / (m + n + d)!
// on the reference simplex (volume 1/d!), and dB_beta^n/dxi_a =
// n (B^{n-1}_{beta - e_a} - B^{n-1}_{beta - e_0}).

// Error-free transformations (Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005): a + b = s + e and a * b = p + e exactly.  The rounded
// product passes through a volatile so that no compiler contraction fuses it
// into a later addition; std::fma is correctly rounded on every target, so
// both transformations are exact on every host.
static inline void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    const double z = s - a;
    e = (a - (s - z)) + (b - z);
}
static inline void two_prod(double a, double b, double& p, double& e) {
    volatile double pv = a * b;
    p = pv;
    e = std::fma(a, b, -p);
}

// multi-indices (beta_0, ..., beta_d) of total degree n, in the order of
// RefElement::alpha
static std::vector<std::array<int, 4>> lattice_indices(int d, int n) {
    std::vector<std::array<int, 4>> out;
    if (d == 2) {
        for (int j = 0; j <= n; ++j)
            for (int i = 0; i <= n - j; ++i) out.push_back({n - i - j, i, j, 0});
    } else {
        for (int l = 0; l <= n; ++l)
            for (int j = 0; j <= n - l; ++j)
                for (int i = 0; i <= n - l - j; ++i) out.push_back({n - i - j - l, i, j, l});
    }
    return out;
}

// multinomial n! / (b_0! ... b_d!) for |b| = n, exact in 64-bit integers
// (every partial product is itself a multinomial coefficient)
static long long multinomial(const std::array<int, 4>& b, int d) {
    long long r = 1;
    int m = 0;
    for (int c = 0; c <= d; ++c)
        for (int t = 1; t <= b[c]; ++t) r = r * (++m) / t;
    return r;
}

// Bernstein coefficients of the degree-k Lagrange basis of `e`: row i holds
// phi_i = sum_b C[i][b] B_b, b in lattice_indices(d, k) order.  C = G^-T for
// the collocation matrix G[node][b] = B_b(node) = (k!/b!) prod_c alpha_c^b_c
// / k^k.  k^k G is an integer matrix with entries at most k^k (the
// multinomial theorem), exact in double up to k = 10, so it is inverted
// exactly as given: Gauss-Jordan with partial pivoting (cond below 4e3 up to
// k = 10 in 3D), then iterative refinement.
// G^-1 for an n x n matrix G given exactly: Gauss-Jordan with partial
// pivoting, then `steps` steps of iterative refinement X += X (I - G X) with
// the residual from compensated dot products, each of which multiplies the
// error by about cond(G) eps (so cond(G) well below 1/eps is needed).
static std::vector<double> invert_refined(const std::vector<double>& G, int n, int steps) {
    std::vector<double> A((size_t)n * 2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[(size_t)i * 2 * n + j] = G[(size_t)i * n + j];
        A[(size_t)i * 2 * n + n + i] = 1.0;
    }
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * 2 * n + c]) > std::fabs(A[(size_t)p * 2 * n + c])) p = r;
        if (p != c)
            for (int j = 0; j < 2 * n; ++j) std::swap(A[(size_t)p * 2 * n + j], A[(size_t)c * 2 * n + j]);
        const double piv = A[(size_t)c * 2 * n + c];
        if (piv == 0) throw std::runtime_error("singular collocation matrix of a reference element");
        for (int j = 0; j < 2 * n; ++j) A[(size_t)c * 2 * n + j] /= piv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * 2 * n + c];
            if (f == 0) continue;
            for (int j = 0; j < 2 * n; ++j) A[(size_t)r * 2 * n + j] -= f * A[(size_t)c * 2 * n + j];
        }
    }
    std::vector<double> X((size_t)n * n), R((size_t)n * n);
    for (int b = 0; b < n; ++b)
        for (int i = 0; i < n; ++i) X[(size_t)b * n + i] = A[(size_t)b * 2 * n + n + i];
    for (int step = 0; step < steps; ++step) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double sum = i == j ? 1.0 : 0.0, err = 0;
                for (int l = 0; l < n; ++l) {
                    double p, pe, se;
                    two_prod(-G[(size_t)i * n + l], X[(size_t)l * n + j], p, pe);
                    two_sum(sum, p, sum, se);
                    err += pe + se;
                }
                R[(size_t)i * n + j] = sum + err;
            }
        std::vector<double> Xn(X);
        for (int b = 0; b < n; ++b)
            for (int j = 0; j < n; ++j) {
                double corr = 0;
                for (int l = 0; l < n; ++l) corr += X[(size_t)b * n + l] * R[(size_t)l * n + j];
                Xn[(size_t)b * n + j] += corr;
            }
        X.swap(Xn);
    }
    return X;
}

// Bernstein coefficients of the degree-k Lagrange basis of `e`: row i holds
// phi_i = sum_b C[i][b] B_b, b in lattice_indices(d, k) order.  C = G^-T for
// the collocation matrix G[node][b] = B_b(node) = (k!/b!) prod_c alpha_c^b_c
// / k^k.  k^k G is an integer matrix with entries at most k^k (the
// multinomial theorem), exact in double up to k = 10, so it is inverted
// exactly as given (cond below 4e3 up to k = 10 in 3D).
static std::vector<double> lagrange_in_bernstein(const RefElement& e) {
    const int d = e.d, k = e.k, n = e.nb;
    const auto B = lattice_indices(d, k);
    long long kk = 1;
    for (int c = 0; c < k; ++c) kk *= k;
    if (kk > (1LL << 53)) throw std::runtime_error("reference element degree too high for exact collocation");
    std::vector<double> G((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int b = 0; b < n; ++b) {
            long long num = 1;
            for (int c = 0; c <= d; ++c)
                for (int t = 0; t < B[b][c]; ++t) num *= e.alpha[i][c];
            G[(size_t)i * n + b] = (double)(multinomial(B[b], d) * num);   // at most k^k
        }
    const std::vector<double> X = invert_refined(G, n, 2);
    std::vector<double> C((size_t)n * n);
    for (int b = 0; b < n; ++b)
        for (int i = 0; i < n; ++i) C[(size_t)i * n + b] = X[(size_t)b * n + i] * (double)kk;
    return C;
}

// W[b][g] = int B_b^m B_g^n over the reference d-simplex, as an unevaluated
// pair hi + lo: with s = b + g,
//   W = mult(m; b) mult(n; g) / (mult(m + n; s) (m+n+1) ... (m+n+d)),
// numerator and denominator exact in double (below 2^53 up to m = n = 10),
// so hi is the rounded quotient and lo its exact remainder divided out
struct PairMatrix {
    std::vector<double> hi, lo;
};
static PairMatrix bernstein_products(int d, int m, int n) {
    const auto Bm = lattice_indices(d, m), Bn = lattice_indices(d, n);
    PairMatrix W;
    W.hi.resize(Bm.size() * Bn.size());
    W.lo.resize(Bm.size() * Bn.size());
    long long tail = 1;
    for (int t = 1; t <= d; ++t) tail *= m + n + t;
    for (size_t b = 0; b < Bm.size(); ++b)
        for (size_t g = 0; g < Bn.size(); ++g) {
            std::array<int, 4> s{};
            for (int c = 0; c <= d; ++c) s[c] = Bm[b][c] + Bn[g][c];
            const long long num = multinomial(Bm[b], d) * multinomial(Bn[g], d);
            const long long den = multinomial(s, d) * tail;
            if (num > (1LL << 53) || den > (1LL << 53))
                throw std::runtime_error("reference element degree too high for exact Bernstein integrals");
            const double hi = (double)num / (double)den;
            const double rem = std::fma(-hi, (double)den, (double)num);   // exact: num - hi den
            W.hi[b * Bn.size() + g] = hi;
            W.lo[b * Bn.size() + g] = rem / (double)den;
        }
    return W;
}

// PW[r][y] = sum_x P[r][x] W[x][y] (P: rp x nx, W: nx x ny) as pairs hi + lo,
// compensated: the Lagrange coefficients in P carry signs, and plain double
// sums lose three to four digits to cancellation at k = 10
static PairMatrix left_product(const std::vector<double>& P, int rp, int nx, const PairMatrix& W, int ny) {
    PairMatrix PW;
    PW.hi.resize((size_t)rp * ny);
    PW.lo.resize((size_t)rp * ny);
    for (int r = 0; r < rp; ++r)
        for (int y = 0; y < ny; ++y) {
            double sum = 0, err = 0;
            for (int x = 0; x < nx; ++x) {
                const double a = P[(size_t)r * nx + x];
                double p, pe, se;
                two_prod(a, W.hi[(size_t)x * ny + y], p, pe);
                two_sum(sum, p, sum, se);
                err += pe + se + a * W.lo[(size_t)x * ny + y];
            }
            two_sum(sum, err, PW.hi[(size_t)r * ny + y], PW.lo[(size_t)r * ny + y]);
        }
    return PW;
}

// out[r][c] = sum_y PW[r][y] Q[c][y]  (Q: cq x ny), compensated
static std::vector<double> right_product(const PairMatrix& PW, int rp, const std::vector<double>& Q, int cq, int ny) {
    std::vector<double> out((size_t)rp * cq);
    for (int r = 0; r < rp; ++r)
        for (int c = 0; c < cq; ++c) {
            double sum = 0, err = 0;
            for (int y = 0; y < ny; ++y) {
                const double q = Q[(size_t)c * ny + y];
                double p, pe, se;
                two_prod(PW.hi[(size_t)r * ny + y], q, p, pe);
                two_sum(sum, p, sum, se);
                err += pe + se + PW.lo[(size_t)r * ny + y] * q;
            }
            out[(size_t)r * cq + c] = sum + err;
        }
    return out;
}

// phi_i(xi) = sum_b bcoef[i][b] B_b(lambda(xi)), compensated: the Bernstein
// values are nonnegative and sum to one, so the result is accurate to a few
// units of the last place at any degree (the monomial expansion in coef
// loses digits with the degree: 1.7e-10 for P9 at lattice points)
void RefElement::eval(const double* xi, double* out) const {
    double lam[4] = {1.0, 0.0, 0.0, 0.0};
    for (int c = 0; c < d; ++c) {
        lam[c + 1] = xi[c];
        lam[0] -= xi[c];
    }
    double pw[4][11];                 // lambda_c^e, e <= k <= 10
    for (int c = 0; c <= d; ++c) {
        pw[c][0] = 1.0;
        for (int e2 = 1; e2 <= k; ++e2) pw[c][e2] = pw[c][e2 - 1] * lam[c];
    }
    double bv[320];                   // up to P_10 in 3D (286 basis functions)
    for (int b = 0; b < nb; ++b) {
        double v = (double)multinomial(alpha[b], d);
        for (int c = 0; c <= d; ++c) v *= pw[c][alpha[b][c]];
        bv[b] = v;
    }
    for (int i = 0; i < nb; ++i) {
        double sum = 0, err = 0;
        for (int b = 0; b < nb; ++b) {
            double p, pe, se;
            two_prod(bcoef[(size_t)i * nb + b], bv[b], p, pe);
            two_sum(sum, p, sum, se);
            err += pe + se;
        }
        out[i] = sum + err;
    }
}

void RefTensors::init(const RefElement& v, const RefElement& q) {
    d = v.d;
    nb = v.nb;
    nq = q.nb;
    const int k = v.k, kq = q.k;
    const std::vector<double>& Cv = v.bcoef;
    const std::vector<double>& Cp = q.bcoef;
    // derivative coefficients in the degree k - 1 Bernstein basis:
    // dphi_i/dxi_a = sum_g D_a[i][g] B_g^{k-1}
    const auto Bk = lattice_indices(d, k), Bk1 = lattice_indices(d, k - 1);
    const int n1 = (int)Bk1.size();
    // position in Bk (RefElement order) of a degree-k multi-index, from (beta_1, .., beta_d)
    std::vector<int> pos_k((size_t)(k + 1) * (k + 1) * (d == 3 ? k + 1 : 1), -1);
    auto key = [&](const std::array<int, 4>& b) { return (size_t)b[1] + (size_t)(k + 1) * (b[2] + (size_t)(k + 1) * b[3]); };
    for (int x = 0; x < (int)Bk.size(); ++x) pos_k[key(Bk[x])] = x;
    auto index_k = [&](const std::array<int, 4>& b) { return pos_k[key(b)]; };
    std::vector<int> up0(n1), upa((size_t)d * n1);
    for (int g = 0; g < n1; ++g) {
        auto b = Bk1[g];
        b[0] += 1;
        up0[g] = index_k(b);
        for (int a = 0; a < d; ++a) {
            auto c = Bk1[g];
            c[a + 1] += 1;
            upa[(size_t)a * n1 + g] = index_k(c);
        }
    }
    std::vector<std::vector<double>> D(d, std::vector<double>((size_t)nb * n1));
    for (int a = 0; a < d; ++a)
        for (int i = 0; i < nb; ++i)
            for (int g = 0; g < n1; ++g)
                D[a][(size_t)i * n1 + g] = k * (Cv[(size_t)i * nb + upa[(size_t)a * n1 + g]] - Cv[(size_t)i * nb + up0[g]]);
    const PairMatrix Wkk = bernstein_products(d, k, k), W11 = bernstein_products(d, k - 1, k - 1),
                     Wq1 = bernstein_products(d, kq, k - 1);
    // S[a][b] = D_a W D_b^T; S[b][a] is its transpose
    S.assign((size_t)d * d * nb * nb, 0.0);
    for (int a = 0; a < d; ++a) {
        const PairMatrix DW = left_product(D[a], nb, n1, W11, n1);
        for (int b = a; b < d; ++b) {
            const std::vector<double> Sab = right_product(DW, nb, D[b], nb, n1);
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j) {
                    S[(((size_t)a * d + b) * nb + i) * nb + j] = Sab[(size_t)i * nb + j];
                    S[(((size_t)b * d + a) * nb + j) * nb + i] = Sab[(size_t)i * nb + j];
                }
        }
    }
    Cq.assign((size_t)d * nq * nb, 0.0);
    const PairMatrix CW = left_product(Cp, nq, nq, Wq1, n1);
    for (int a = 0; a < d; ++a) {
        const std::vector<double> Ca = right_product(CW, nq, D[a], nb, n1);
        std::copy(Ca.begin(), Ca.end(), Cq.begin() + (size_t)a * nq * nb);
    }
    M = right_product(left_product(Cv, nb, nb, Wkk, nb), nb, Cv, nb, nb);
    // int B_b^kq = kq! / (kq + d)! = 1 / ((kq + 1) ... (kq + d)) for every b
    qint.assign(nq, 0.0);
    double tail = 1.0;
    for (int t = 1; t <= d; ++t) tail *= kq + t;
    for (int p = 0; p < nq; ++p) {
        double sum = 0, err = 0;
        for (int b = 0; b < nq; ++b) {
            double se;
            two_sum(sum, Cp[(size_t)p * nq + b], sum, se);
            err += se;
        }
        qint[p] = (sum + err) / tail;
    }
}

CSR transpose(const CSR& a) {
    CSR t;
    t.nr = a.ncol;
    t.ncol = a.nr;
    const int T = chunk_count(a.nr);
    std::vector<std::vector<int>> hist(T, std::vector<int>(a.ncol + 1, 0));
    Pool::get().run(T, [&](int th) {
        const int lo = (int)((long long)a.nr * th / T), hi = (int)((long long)a.nr * (th + 1) / T);
        auto& hh = hist[th];
        for (int p = a.rp[lo]; p < a.rp[hi]; ++p) hh[a.ci[p]]++;
    });
    // column c of thread th starts after all of column c's entries from
    // threads < th: rows stay in increasing order within every column
    t.rp.assign(t.nr + 1, 0);
    std::vector<std::vector<int>> start(T, std::vector<int>(a.ncol));
    long long run = 0;
    for (int col = 0; col < a.ncol; ++col) {
        t.rp[col] = (int)run;
        for (int th = 0; th < T; ++th) {
            start[th][col] = (int)run;
            run += hist[th][col];
        }
    }
    t.rp[t.nr] = index_total(run, "transposed matrix");
    t.ci.resize(run);
    t.v.resize(run);
    Pool::get().run(T, [&](int th) {
        const int lo = (int)((long long)a.nr * th / T), hi = (int)((long long)a.nr * (th + 1) / T);
        auto& st = start[th];
        for (int r = lo; r < hi; ++r)
            for (int p = a.rp[r]; p < a.rp[r + 1]; ++p) {
                const int q = st[a.ci[p]]++;
                t.ci[q] = r;
                t.v[q] = a.v[p];
            }
    });
    return t;
}

// ------------------------------------------------------------------ spaces --
struct Topology {
    int d = 0, ne = 0, nf = 0;
    std::vector<int> cell_edge;             // [nc][d==2 ? 3 : 6], local edge order of kEdges
    std::vector<int> cell_face;             // [nc][4] (3D): face opposite local vertex i
    std::vector<unsigned char> bvert, bedge, bface;   // on the boundary, by vertex / edge / face id
    std::vector<int> v2c_off, v2c;          // vertex -> cells
    int max_valence = 0;                    // most cells around one vertex
};

// local vertex pairs of the edges of a simplex (2D uses the first three
// entries of the triangle table)
static const int kEdges2[3][2] = {{0, 1}, {0, 2}, {1, 2}};
static const int kEdges3[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

static inline int local_edge(int d, int i, int j) {
    if (i > j) std::swap(i, j);
    if (d == 2) return i == 0 ? j - 1 : 2;
    return i == 0 ? j - 1 : (i == 1 ? j + 1 : 5);
}

static inline uint64_t face_key(int a, int b, int c, int nv) {
    int t[3] = {a, b, c};
    std::sort(t, t + 3);
    return ((uint64_t)t[0] * (uint64_t)nv + (uint64_t)t[1]) * (uint64_t)nv + (uint64_t)t[2];
}

static void build_topology(const Mesh& m, Topology& T) {
    const int d = m.d, nvpc = d + 1, nle = d == 2 ? 3 : 6;
    PhaseClock pc("topology");
    T.d = d;
    // vertex -> cells (cells in increasing index)
    T.v2c_off.assign(m.nv + 1, 0);
    for (int x : m.C) T.v2c_off[x + 1]++;
    T.max_valence = 0;
    for (int i = 0; i < m.nv; ++i) {
        T.max_valence = std::max(T.max_valence, T.v2c_off[i + 1]);
        T.v2c_off[i + 1] += T.v2c_off[i];
    }
    T.v2c.resize(m.C.size());
    {
        std::vector<int> fill(T.v2c_off.begin(), T.v2c_off.end() - 1);
        for (int e = 0; e < m.nc; ++e)
            for (int i = 0; i < nvpc; ++i) T.v2c[fill[m.C[(size_t)e * nvpc + i]]++] = e;
    }
    // edges numbered vertex by vertex: edge (a, b), a < b, is the rank of b
    // among the sorted distinct neighbours w > a of a (over a's cells),
    // offset by the counts of the vertices before a.  Built in parallel
    // without hashing; only the identity of the ids matters downstream.
    pc.lap("vertex->cells");
    std::vector<int> nbr_off(m.nv + 1, 0);
    auto upper_neighbours = [&](int a, std::vector<int>& w) {
        w.clear();
        for (int x = T.v2c_off[a]; x < T.v2c_off[a + 1]; ++x) {
            const int* v = &m.C[(size_t)T.v2c[x] * nvpc];
            for (int i = 0; i < nvpc; ++i)
                if (v[i] > a) w.push_back(v[i]);
        }
        std::sort(w.begin(), w.end());
        w.erase(std::unique(w.begin(), w.end()), w.end());
    };
    parallel_for(m.nv, [&](int lo, int hi, int) {
        std::vector<int> w;
        for (int a = lo; a < hi; ++a) {
            upper_neighbours(a, w);
            nbr_off[a + 1] = (int)w.size();
        }
    }, 64, 4);
    for (int a = 0; a < m.nv; ++a) nbr_off[a + 1] += nbr_off[a];
    std::vector<int> nbr(nbr_off[m.nv]);
    parallel_for(m.nv, [&](int lo, int hi, int) {
        std::vector<int> w;
        for (int a = lo; a < hi; ++a) {
            upper_neighbours(a, w);
            std::copy(w.begin(), w.end(), nbr.begin() + nbr_off[a]);
        }
    }, 64, 4);
    pc.lap("edge lists");
    T.cell_edge.resize((size_t)m.nc * nle);
    parallel_for(m.nc, [&](int lo, int hi, int) {
        for (int e = lo; e < hi; ++e) {
            const int* v = &m.C[(size_t)e * nvpc];
            for (int t = 0; t < nle; ++t) {
                const int i = d == 2 ? kEdges2[t][0] : kEdges3[t][0], j = d == 2 ? kEdges2[t][1] : kEdges3[t][1];
                const int a = std::min(v[i], v[j]), b = std::max(v[i], v[j]);
                const int* first = nbr.data() + nbr_off[a];
                const int* last = nbr.data() + nbr_off[a + 1];
                T.cell_edge[(size_t)e * nle + t] = nbr_off[a] + (int)(std::lower_bound(first, last, b) - first);
            }
        }
    }, 256, 4);
    T.ne = nbr_off[m.nv];
    pc.lap("cell edges");
    std::vector<int> facet_count;
    if (d == 3) {
        T.cell_face.resize((size_t)m.nc * 4);
        std::unordered_map<uint64_t, int> fid;
        fid.reserve((size_t)m.nc * 2);
        for (int e = 0; e < m.nc; ++e) {
            const int* v = &m.C[(size_t)e * 4];
            for (int i = 0; i < 4; ++i) {
                int f[3], t = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != i) f[t++] = v[j];
                auto ins = fid.emplace(face_key(f[0], f[1], f[2], m.nv), (int)fid.size());
                T.cell_face[(size_t)e * 4 + i] = ins.first->second;
            }
        }
        T.nf = (int)fid.size();
        facet_count.assign(T.nf, 0);
        for (int x : T.cell_face) facet_count[x]++;
    } else {
        facet_count.assign(T.ne, 0);
        for (int x : T.cell_edge) facet_count[x]++;
    }
    pc.lap("faces/facet counts");
    // boundary facets: owned by one cell; mark their vertices, edges, faces
    T.bvert.assign(m.nv, 0);
    T.bedge.assign(T.ne, 0);
    T.bface.assign(T.nf, 0);
    for (int e = 0; e < m.nc; ++e) {
        const int* v = &m.C[(size_t)e * nvpc];
        for (int i = 0; i < nvpc; ++i) {          // facet opposite local vertex i
            const int fidx = d == 3 ? T.cell_face[(size_t)e * 4 + i]
                                    : T.cell_edge[(size_t)e * 3 + local_edge(2, (i + 1) % 3, (i + 2) % 3)];
            if (facet_count[fidx] != 1) continue;
            for (int j = 0; j < nvpc; ++j)
                if (j != i) T.bvert[v[j]] = 1;
            if (d == 2) {
                T.bedge[fidx] = 1;
            } else {
                T.bface[fidx] = 1;
                for (int a = 0; a < 4; ++a)
                    for (int b2 = a + 1; b2 < 4; ++b2)
                        if (a != i && b2 != i) T.bedge[T.cell_edge[(size_t)e * 6 + local_edge(3, a, b2)]] = 1;
            }
        }
    }
    pc.lap("boundary");
}

static int binom(int n, int r) {
    if (r < 0 || r > n) return 0;
    long long b = 1;
    for (int i = 1; i <= r; ++i) b = b * (n - r + i) / i;
    return (int)b;
}

// Continuous space: a node on cell e with multi-index alpha is owned by the
// entity spanned by the vertices with alpha_i > 0; inside that entity it is
// identified by the alpha values listed in increasing global vertex order
// (a composition of k into |S| positive parts).  Nodes are finally
// renumbered in order of first appearance over the cells (locality).
static void build_space(const Mesh& m, const Topology& T, const RefElement& re, bool continuous, Space& S) {
    const int d = m.d, nvpc = d + 1, nb = re.nb, k = re.k;
    S.d = d;
    S.k = k;
    S.nb = nb;
    S.continuous = continuous;
    S.cell_nodes.assign((size_t)m.nc * nb, -1);
    if (!continuous) {
        S.n = m.nc * nb;
        S.X.resize((size_t)S.n * d);
        S.boundary.assign(S.n, 0);
        S.support.resize(S.n);
        S.owner_cell.resize(S.n);
        S.owner_local.resize(S.n);
        parallel_for(m.nc, [&](int lo, int hi, int) {
            for (int e = lo; e < hi; ++e) {
                const int* v = &m.C[(size_t)e * nvpc];
                std::array<int, 4> sup = {-1, -1, -1, -1};
                for (int i = 0; i < nvpc; ++i) sup[i] = v[i];
                std::sort(sup.begin(), sup.begin() + nvpc);
                for (int l = 0; l < nb; ++l) {
                    int id = e * nb + l;
                    S.cell_nodes[(size_t)e * nb + l] = id;
                    for (int c = 0; c < d; ++c) {
                        double x = 0;
                        for (int i = 0; i < nvpc; ++i) x += re.alpha[l][i] * m.X[(size_t)v[i] * d + c];
                        S.X[(size_t)id * d + c] = x / (k > 0 ? k : 1);
                    }
                    S.support[id] = sup;
                    S.owner_cell[id] = e;
                    S.owner_local[id] = l;
                }
            }
        });
        return;
    }
    PhaseClock pc(continuous ? "space" : "space-dg");
    // rank tables for compositions of k into m positive parts
    std::vector<std::vector<int>> rank(5);
    std::vector<int> nint(5, 0);
    for (int mm = 1; mm <= nvpc; ++mm) {
        nint[mm] = binom(k - 1, mm - 1);
        long long ncode = 1;
        for (int t = 0; t < mm; ++t) ncode *= (k + 1);
        rank[mm].assign(ncode, -1);
        int nr = 0;
        std::vector<int> part(mm, 1);
        // enumerate all compositions by recursion over a simple odometer
        std::function<void(int, int)> rec = [&](int pos, int left) {
            if (pos == mm - 1) {
                if (left >= 1) {
                    part[pos] = left;
                    long long code = 0;
                    for (int t = 0; t < mm; ++t) code = code * (k + 1) + part[t];
                    rank[mm][code] = nr++;
                }
                return;
            }
            for (int v = 1; v <= left - (mm - 1 - pos); ++v) {
                part[pos] = v;
                rec(pos + 1, left - v);
            }
        };
        if (k >= mm) rec(0, k);
    }
    const long long ne = T.ne, nf = T.nf;
    long long base[5] = {0, 0, 0, 0, 0};
    base[1] = 0;
    base[2] = base[1] + (long long)m.nv * nint[1];
    base[3] = base[2] + ne * nint[2];
    if (d == 2) {
        base[4] = 0;
    } else {
        base[4] = base[3] + nf * nint[3];
    }
    long long ntmp = d == 2 ? base[3] + (long long)m.nc * nint[3] : base[4] + (long long)m.nc * nint[4];
    pc.lap("rank tables");
    // entity-based id of every (cell, local node)
    std::vector<int> tmp((size_t)m.nc * nb);
    parallel_for(m.nc, [&](int lo, int hi, int) {
        for (int e = lo; e < hi; ++e) {
            const int* v = &m.C[(size_t)e * nvpc];
            for (int l = 0; l < nb; ++l) {
                int sv[4], sa[4], sl[4], mm = 0;
                for (int i = 0; i < nvpc; ++i)
                    if (re.alpha[l][i] > 0) { sv[mm] = v[i]; sa[mm] = re.alpha[l][i]; sl[mm] = i; ++mm; }
                for (int a = 1; a < mm; ++a)          // sort by global vertex id
                    for (int b = a; b > 0 && sv[b - 1] > sv[b]; --b) {
                        std::swap(sv[b - 1], sv[b]); std::swap(sa[b - 1], sa[b]); std::swap(sl[b - 1], sl[b]);
                    }
                long long code = 0;
                for (int t = 0; t < mm; ++t) code = code * (k + 1) + sa[t];
                int r = rank[mm][code];
                long long eid;
                if (mm == 1) eid = sv[0];
                else if (mm == 2) eid = T.cell_edge[(size_t)e * (d == 2 ? 3 : 6) + local_edge(d, sl[0], sl[1])];
                else if (mm == 3 && d == 3) eid = T.cell_face[(size_t)e * 4 + (6 - sl[0] - sl[1] - sl[2])];
                else eid = e;   // cell interior
                tmp[(size_t)e * nb + l] = (int)(base[mm] + eid * nint[mm] + r);
            }
        }
    }, 128, 4);
    // renumber by first appearance: first[x] = least position of id x, the
    // first positions in increasing order get 0, 1, 2, ...
    pc.lap("entity ids");
    const long long ntot = (long long)tmp.size();
    fvec<int> first(ntmp);
    parallel_for((int)ntmp, [&](int lo, int hi, int) { std::fill(first.begin() + lo, first.begin() + hi, INT32_MAX); },
                 8192, 4);
    parallel_for((int)ntot, [&](int lo, int hi, int) {
        for (int t = lo; t < hi; ++t) {
            int* f = &first[tmp[t]];
            int cur = __atomic_load_n(f, __ATOMIC_RELAXED);
            while (t < cur && !__atomic_compare_exchange_n(f, &cur, t, true, __ATOMIC_RELAXED, __ATOMIC_RELAXED)) {}
        }
    }, 4096, 4);
    fvec<int> isfirst(ntot), rankpos(ntot + 1);
    parallel_for((int)ntot, [&](int lo, int hi, int) {
        for (int t = lo; t < hi; ++t) isfirst[t] = first[tmp[t]] == t;
    }, 4096, 4);
    parallel_scan(isfirst.data(), (int)ntot, rankpos.data());
    pc.lap("first appearance");
    const int n = rankpos[ntot];
    parallel_for((int)ntot, [&](int lo, int hi, int) {
        for (int t = lo; t < hi; ++t) S.cell_nodes[t] = rankpos[first[tmp[t]]];
    }, 4096, 4);
    pc.lap("cell nodes");
    S.n = n;
    // every field of every node is written below, by its first (cell, local
    // node): no serial initialisation
    S.X.resize((size_t)n * d);
    S.boundary.resize(n);
    S.support.resize(n);
    S.owner_cell.resize(n);
    S.owner_local.resize(n);
    // node data from its first (cell, local node)
    parallel_for((int)ntot, [&](int lo, int hi, int) {
        for (int t = lo; t < hi; ++t) {
            if (!isfirst[t]) continue;
            const int e = t / nb, l = t % nb, id = rankpos[t];
            const int* v = &m.C[(size_t)e * nvpc];
            S.owner_cell[id] = e;
            S.owner_local[id] = l;
            for (int c = 0; c < d; ++c) {
                double x = 0;
                for (int i = 0; i < nvpc; ++i) x += re.alpha[l][i] * m.X[(size_t)v[i] * d + c];
                S.X[(size_t)id * d + c] = x / k;
            }
            int sv[4], sl[4], mm = 0;
            for (int i = 0; i < nvpc; ++i)
                if (re.alpha[l][i] > 0) { sv[mm] = v[i]; sl[mm] = i; ++mm; }
            {
                int tmpv[4];
                for (int q = 0; q < mm; ++q) tmpv[q] = sv[q];
                std::sort(tmpv, tmpv + mm);
                for (int q = 0; q < 4; ++q) S.support[id][q] = q < mm ? tmpv[q] : -1;
            }
            bool b;
            if (mm == 1) b = T.bvert[sv[0]];
            else if (mm == 2) b = T.bedge[T.cell_edge[(size_t)e * (d == 2 ? 3 : 6) + local_edge(d, sl[0], sl[1])]];
            else if (mm == 3 && d == 3) b = T.bface[T.cell_face[(size_t)e * 4 + (6 - sl[0] - sl[1] - sl[2])]];
            else b = false;
            S.boundary[id] = b;
        }
    }, 4096, 4);
    pc.lap("node data");
}

// --------------------------------------------------------------- assembly --
struct CellGeom {
    double detabs;
    double Jinv[9];   // [a][c] = d xi_a / d x_c
};

static CellGeom cell_geom(const Mesh& m, int e) {
    const int d = m.d;
    const int* v = &m.C[(size_t)e * (d + 1)];
    double J[9];
    for (int c = 0; c < d; ++c)
        for (int a = 0; a < d; ++a) J[c * d + a] = m.X[(size_t)v[a + 1] * d + c] - m.X[(size_t)v[0] * d + c];
    CellGeom g;
    if (d == 2) {
        double det = J[0] * J[3] - J[1] * J[2];
        g.detabs = std::fabs(det);
        // Jinv[a][c]
        g.Jinv[0] = J[3] / det;  g.Jinv[1] = -J[1] / det;
        g.Jinv[2] = -J[2] / det; g.Jinv[3] = J[0] / det;
    } else {
        double a = J[0], b = J[1], c = J[2], dd = J[3], e2 = J[4], f = J[5], gg = J[6], h = J[7], i = J[8];
        double A = e2 * i - f * h, B = -(dd * i - f * gg), Cc = dd * h - e2 * gg;
        double det = a * A + b * B + c * Cc;
        g.detabs = std::fabs(det);
        double inv[9] = {A, -(b * i - c * h), b * f - c * e2,
                         B, a * i - c * gg, -(a * f - c * dd),
                         Cc, -(a * h - b * gg), a * e2 - b * dd};
        for (int t = 0; t < 9; ++t) g.Jinv[t] = inv[t] / det;
    }
    return g;
}

// node -> (cell, local index) adjacency
static void node_cells(const Space& S, int nc, std::vector<int>& off, std::vector<int>& adj) {
    // (cells in increasing index for every node)
    invert_index(S.cell_nodes.data(), (long long)nc * S.nb, S.n, off, adj);
}

// DoF maps and adjacency a device assembly needs (no matrices).
static void prepare_level(const Mesh& m, Level& L, const RefTensors& RT) {
    const int d = m.d, nq = L.Q.nb, nc = m.nc;
    const Space &V = L.V, &Q = L.Q;
    PhaseClock pc("prepare");
    L.vfree.assign(V.n, -1);
    int nVf = 0;
    for (int i = 0; i < V.n; ++i)
        if (!V.boundary[i]) L.vfree[i] = nVf++;
    L.nVf = nVf;
    L.nQ = Q.n;
    L.n_free = d * nVf + Q.n;
    pc.lap("free numbering");
    // (the node -> cell incidence lists a device assembly reads are built on
    // the device from the cell-node maps)
    std::vector<double> det(nc);
    L.cell_center.resize((size_t)nc * d);
    parallel_for(nc, [&](int lo, int hi, int) {
        for (int e = lo; e < hi; ++e) {
            det[e] = cell_geom(m, e).detabs;
            for (int cc = 0; cc < d; ++cc) {
                double s = 0;
                for (int i = 0; i <= d; ++i) s += m.X[(size_t)m.C[(size_t)e * (d + 1) + i] * d + cc];
                L.cell_center[(size_t)e * d + cc] = s / (d + 1);
            }
        }
    }, 1024);
    // int psi_q: the contributions of the incident cells in increasing cell
    // order (a node occurs once per cell)
    L.pint.assign(Q.n, 0.0);
    for (int e = 0; e < nc; ++e)
        for (int l = 0; l < nq; ++l) L.pint[Q.cell_nodes[(size_t)e * nq + l]] += det[e] * RT.qint[l];
    pc.lap("geometry, int psi");
}

static void assemble_level(const Mesh& m, Level& L, const RefTensors& RT, const std::vector<double>& nu,
                           bool with_load) {
    const int d = m.d, nb = L.V.nb, nq = L.Q.nb, nc = m.nc;
    const Space &V = L.V, &Q = L.Q;
    // element matrices: stiffness (scaled by nu_e) and divergence coupling
    fvec<double> Se((size_t)nc * nb * nb), Ce((size_t)nc * nq * nb * d), Me((size_t)nc * nb * nb);
    fvec<double> qe((size_t)nc * nq);
    parallel_for(nc, [&](int lo, int hi, int) {
        for (int e = lo; e < hi; ++e) {
            CellGeom g = cell_geom(m, e);
            double G[9];
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int c = 0; c < d; ++c) s += g.Jinv[a * d + c] * g.Jinv[b * d + c];
                    G[a * d + b] = s;
                }
            double w = g.detabs * (nu.empty() ? 1.0 : nu[e]);
            for (int i = 0; i < nb; ++i)
                for (int j = 0; j < nb; ++j) {
                    double s = 0;
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) s += G[a * d + b] * RT.S[(((size_t)a * d + b) * nb + i) * nb + j];
                    Se[((size_t)e * nb + i) * nb + j] = w * s;
                    Me[((size_t)e * nb + i) * nb + j] = g.detabs * RT.M[(size_t)i * nb + j];
                }
            // C[p][j][c] = -|det J| sum_a Jinv[a][c] Cq[a][p][j]
            for (int p = 0; p < nq; ++p) {
                qe[(size_t)e * nq + p] = g.detabs * RT.qint[p];
                for (int j = 0; j < nb; ++j)
                    for (int c = 0; c < d; ++c) {
                        double s = 0;
                        for (int a = 0; a < d; ++a) s += g.Jinv[a * d + c] * RT.Cq[((size_t)a * nq + p) * nb + j];
                        Ce[(((size_t)e * nq + p) * nb + j) * d + c] = -g.detabs * s;
                    }
            }
        }
    });
    // free numbering
    L.vfree.assign(V.n, -1);
    int nVf = 0;
    for (int i = 0; i < V.n; ++i)
        if (!V.boundary[i]) L.vfree[i] = nVf++;
    L.nVf = nVf;
    L.nQ = Q.n;
    L.n_free = d * nVf + Q.n;
    node_cells(V, nc, L.voff, L.vadj);
    node_cells(Q, nc, L.qoff, L.qadj);
    const std::vector<int>&voff = L.voff, &vadj = L.vadj, &qoff = L.qoff, &qadj = L.qadj;
    // pressure integrals
    L.pint.assign(Q.n, 0.0);
    for (int e = 0; e < nc; ++e)
        for (int p = 0; p < nq; ++p) L.pint[Q.cell_nodes[(size_t)e * nq + p]] += qe[(size_t)e * nq + p];
    // --- row patterns, per velocity node and per pressure node
    // velocity node i: free velocity neighbours (sorted by free index),
    // Dirichlet velocity neighbours, pressure neighbours
    const int T = Pool::get().size();
    std::vector<std::vector<int>> stampV(T, std::vector<int>(V.n, -1)), stampQ(T, std::vector<int>(Q.n, -1));
    auto by_free = [&](int a, int b) { return L.vfree[a] < L.vfree[b]; };
    FlatLists vnb = build_lists(V.n, [&](int i, std::vector<int>& out, int t) {
        auto& sv = stampV[t];
        size_t s0 = out.size();
        for (int a = voff[i]; a < voff[i + 1]; ++a) {
            int e = vadj[a] / nb;
            for (int l = 0; l < nb; ++l) {
                int j = V.cell_nodes[(size_t)e * nb + l];
                if (sv[j] == i || L.vfree[j] < 0) continue;
                sv[j] = i;
                out.push_back(j);
            }
        }
        std::sort(out.begin() + s0, out.end(), by_free);
    });
    for (auto& s : stampV) std::fill(s.begin(), s.end(), -1);
    FlatLists vdn = build_lists(V.n, [&](int i, std::vector<int>& out, int t) {
        auto& sv = stampV[t];
        size_t s0 = out.size();
        for (int a = voff[i]; a < voff[i + 1]; ++a) {
            int e = vadj[a] / nb;
            for (int l = 0; l < nb; ++l) {
                int j = V.cell_nodes[(size_t)e * nb + l];
                if (sv[j] == i || L.vfree[j] >= 0) continue;
                sv[j] = i;
                out.push_back(j);
            }
        }
        std::sort(out.begin() + s0, out.end());
    });
    FlatLists vqn = build_lists(V.n, [&](int i, std::vector<int>& out, int t) {
        auto& sq = stampQ[t];
        size_t s0 = out.size();
        for (int a = voff[i]; a < voff[i + 1]; ++a) {
            int e = vadj[a] / nb;
            for (int l = 0; l < nq; ++l) {
                int q = Q.cell_nodes[(size_t)e * nq + l];
                if (sq[q] == i) continue;
                sq[q] = i;
                out.push_back(q);
            }
        }
        std::sort(out.begin() + s0, out.end());
    });
    for (auto& s : stampV) std::fill(s.begin(), s.end(), -1);
    FlatLists qvn = build_lists(Q.n, [&](int q, std::vector<int>& out, int t) {
        auto& sv = stampV[t];
        size_t s0 = out.size();
        for (int a = qoff[q]; a < qoff[q + 1]; ++a) {
            int e = qadj[a] / nq;
            for (int l = 0; l < nb; ++l) {
                int j = V.cell_nodes[(size_t)e * nb + l];
                if (sv[j] == q || L.vfree[j] < 0) continue;
                sv[j] = q;
                out.push_back(j);
            }
        }
        std::sort(out.begin() + s0, out.end(), by_free);
    });
    for (auto& s : stampV) std::fill(s.begin(), s.end(), -1);
    FlatLists qdn = build_lists(Q.n, [&](int q, std::vector<int>& out, int t) {
        auto& sv = stampV[t];
        size_t s0 = out.size();
        for (int a = qoff[q]; a < qoff[q + 1]; ++a) {
            int e = qadj[a] / nq;
            for (int l = 0; l < nb; ++l) {
                int j = V.cell_nodes[(size_t)e * nb + l];
                if (sv[j] == q || L.vfree[j] >= 0) continue;
                sv[j] = q;
                out.push_back(j);
            }
        }
        std::sort(out.begin() + s0, out.end());
    });
    // --- CSR offsets: rows [comp c free velocity nodes...], then pressure
    const int n = L.n_free;
    std::vector<int> vrow(nVf);   // free index -> node
    for (int i = 0; i < V.n; ++i)
        if (L.vfree[i] >= 0) vrow[L.vfree[i]] = i;
    CSR& K = L.K;
    K.nr = K.ncol = n;
    K.rp.assign(n + 1, 0);
    CSR& KD = L.KfD;
    KD.nr = n;
    KD.ncol = d * V.n;
    KD.rp.assign(n + 1, 0);
    for (int c = 0; c < d; ++c)
        for (int f = 0; f < nVf; ++f) {
            int i = vrow[f];
            K.rp[c * nVf + f + 1] = vnb.size(i) + vqn.size(i);
            KD.rp[c * nVf + f + 1] = vdn.size(i);
        }
    for (int q = 0; q < Q.n; ++q) {
        K.rp[d * nVf + q + 1] = d * qvn.size(q);
        KD.rp[d * nVf + q + 1] = d * qdn.size(q);
    }
    {
        long long sk = 0, sd = 0;
        for (int r = 0; r < n; ++r) {
            sk += K.rp[r + 1];
            sd += KD.rp[r + 1];
            K.rp[r + 1] = index_total(sk, "level operator");
            KD.rp[r + 1] = index_total(sd, "Dirichlet columns of the operator");
        }
    }
    K.ci.resize(K.rp[n]);
    K.v.resize(K.rp[n]);
    KD.ci.resize(KD.rp[n]);
    KD.v.resize(KD.rp[n]);
    // --- values: velocity rows
    std::vector<std::vector<int>> posV(T, std::vector<int>(V.n, -1)), posQ(T, std::vector<int>(Q.n, -1));
    parallel_for(nVf, [&](int lo, int hi, int t) {
        auto& pv = posV[t];
        auto& pq = posQ[t];
        for (int f = lo; f < hi; ++f) {
            int i = vrow[f];
            const int* a = vnb.begin(i);
            const int* b = vqn.begin(i);
            const int* dn = vdn.begin(i);
            const int nvv = vnb.size(i), nbq = vqn.size(i), ndd = vdn.size(i);
            for (int s = 0; s < nvv; ++s) pv[a[s]] = s;
            for (int s = 0; s < ndd; ++s) pv[dn[s]] = s;
            for (int s = 0; s < nbq; ++s) pq[b[s]] = nvv + s;
            for (int c = 0; c < d; ++c) {
                int r = c * nVf + f;
                int* ci = &K.ci[K.rp[r]];
                double* vv = &K.v[K.rp[r]];
                for (int s = 0; s < nvv; ++s) ci[s] = c * nVf + L.vfree[a[s]];
                for (int s = 0; s < nbq; ++s) ci[nvv + s] = d * nVf + b[s];
                for (int s = 0; s < nvv + nbq; ++s) vv[s] = 0.0;
                int* dci = &KD.ci[KD.rp[r]];
                double* dv = &KD.v[KD.rp[r]];
                for (int s = 0; s < ndd; ++s) dci[s] = c * V.n + dn[s];
                for (int s = 0; s < ndd; ++s) dv[s] = 0.0;
                for (int x = voff[i]; x < voff[i + 1]; ++x) {
                    int e = vadj[x] / nb, la = vadj[x] % nb;
                    const double* se = &Se[((size_t)e * nb + la) * nb];
                    for (int l = 0; l < nb; ++l) {
                        int j = V.cell_nodes[(size_t)e * nb + l];
                        if (L.vfree[j] >= 0) vv[pv[j]] += se[l];
                        else dv[pv[j]] += se[l];
                    }
                    for (int p = 0; p < nq; ++p) {
                        int q = Q.cell_nodes[(size_t)e * nq + p];
                        vv[pq[q]] += Ce[(((size_t)e * nq + p) * nb + la) * d + c];
                    }
                }
            }
        }
    });
    // --- values: pressure rows (columns: comp 0 free, comp 1 free, ...)
    parallel_for(Q.n, [&](int lo, int hi, int t) {
        auto& pv = posV[t];
        for (int q = lo; q < hi; ++q) {
            const int* a = qvn.begin(q);
            const int* dn = qdn.begin(q);
            const int nvv = qvn.size(q), ndd = qdn.size(q);
            for (int s = 0; s < nvv; ++s) pv[a[s]] = s;
            for (int s = 0; s < ndd; ++s) pv[dn[s]] = s;
            int r = d * nVf + q;
            int* ci = &K.ci[K.rp[r]];
            double* vv = &K.v[K.rp[r]];
            int* dci = &KD.ci[KD.rp[r]];
            double* dv = &KD.v[KD.rp[r]];
            for (int c = 0; c < d; ++c) {
                for (int s = 0; s < nvv; ++s) ci[c * nvv + s] = c * nVf + L.vfree[a[s]];
                for (int s = 0; s < ndd; ++s) dci[c * ndd + s] = c * V.n + dn[s];
            }
            for (int s = 0; s < d * nvv; ++s) vv[s] = 0.0;
            for (int s = 0; s < d * ndd; ++s) dv[s] = 0.0;
            for (int x = qoff[q]; x < qoff[q + 1]; ++x) {
                int e = qadj[x] / nq, lp = qadj[x] % nq;
                for (int l = 0; l < nb; ++l) {
                    int j = V.cell_nodes[(size_t)e * nb + l];
                    const double* ce = &Ce[(((size_t)e * nq + lp) * nb + l) * d];
                    if (L.vfree[j] >= 0)
                        for (int c = 0; c < d; ++c) vv[c * nvv + pv[j]] += ce[c];
                    else
                        for (int c = 0; c < d; ++c) dv[c * ndd + pv[j]] += ce[c];
                }
            }
        }
    });
    // --- scalar mass matrix on all velocity nodes (for F = M f); only the
    // finest level's load vector is ever formed
    if (!with_load) { L.KfD = CSR(); goto centers; }
    {
    CSR& Mv = L.Mv;
    Mv.nr = Mv.ncol = V.n;
    Mv.rp.assign(V.n + 1, 0);
    {
        long long sm = 0;
        for (int i = 0; i < V.n; ++i) Mv.rp[i + 1] = index_total(sm += vnb.size(i) + vdn.size(i), "mass matrix");
    }
    Mv.ci.resize(Mv.rp[V.n]);
    Mv.v.resize(Mv.rp[V.n]);
    parallel_for(V.n, [&](int lo, int hi, int t) {
        auto& pv = posV[t];
        std::vector<int> cols;
        for (int i = lo; i < hi; ++i) {
            cols.assign(vnb.begin(i), vnb.begin(i) + vnb.size(i));
            cols.insert(cols.end(), vdn.begin(i), vdn.begin(i) + vdn.size(i));
            std::sort(cols.begin(), cols.end());
            for (int s = 0; s < (int)cols.size(); ++s) { pv[cols[s]] = s; Mv.ci[Mv.rp[i] + s] = cols[s]; Mv.v[Mv.rp[i] + s] = 0.0; }
            for (int x = voff[i]; x < voff[i + 1]; ++x) {
                int e = vadj[x] / nb, la = vadj[x] % nb;
                for (int l = 0; l < nb; ++l)
                    Mv.v[Mv.rp[i] + pv[V.cell_nodes[(size_t)e * nb + l]]] += Me[((size_t)e * nb + la) * nb + l];
            }
        }
    });
    }
centers:
    L.cell_center.assign((size_t)nc * d, 0.0);
    for (int e = 0; e < nc; ++e)
        for (int c = 0; c < d; ++c) {
            double s = 0;
            for (int i = 0; i <= d; ++i) s += m.X[(size_t)m.C[(size_t)e * (d + 1) + i] * d + c];
            L.cell_center[(size_t)e * d + c] = s / (d + 1);
        }
}

// Vanka-star patches (Sec. 3.4, Fig. 5): per mesh vertex, the free velocity
// DoFs on all cells around it and the pressure DoFs of its star (TH: nodes
// whose owning entity contains the vertex; SV: all pressure nodes of the
// cells around it).
static void build_patches(const Mesh& m, const Topology& T, Level& L) {
    const int d = m.d, nb = L.V.nb, nq = L.Q.nb;
    PhaseClock pc("patches");
    // per vertex: the free velocity nodes of the cells around it, then the
    // pressure nodes of its star (TH: nodes whose entity has the vertex in
    // its closure) or of those cells (SV), each group sorted and unique
    std::vector<int> NV(m.nv, 0), NP(m.nv, 0);
    // TH: lattice node l of a cell lies on an entity that contains the cell's
    // local vertex i iff its barycentric index alpha_l[i] is positive; SV:
    // every pressure node of the cell belongs to the star
    const int nvpc = d + 1;
    std::vector<unsigned char> in_star((size_t)nvpc * nq, 1);
    if (L.family == 0) {
        const RefElement& rq = reference_element(d, L.Q.k);
        for (int i = 0; i < nvpc; ++i)
            for (int l = 0; l < nq; ++l) in_star[(size_t)i * nq + l] = rq.alpha[l][i] > 0;
    }
    FlatLists lists = build_lists(m.nv, [&](int v, std::vector<int>& out, int) {
        const size_t s0 = out.size();
        for (int a = T.v2c_off[v]; a < T.v2c_off[v + 1]; ++a) {
            const int* cn = &L.V.cell_nodes[(size_t)T.v2c[a] * nb];
            for (int l = 0; l < nb; ++l) {
                const int f = L.vfree[cn[l]];
                if (f >= 0) out.push_back(f);
            }
        }
        sort_unique_tail(out, s0);
        const size_t s1 = out.size();
        for (int a = T.v2c_off[v]; a < T.v2c_off[v + 1]; ++a) {
            const int e = T.v2c[a];
            int i = 0;
            while (i < nvpc && m.C[(size_t)e * nvpc + i] != v) ++i;
            const unsigned char* ok = &in_star[(size_t)std::min(i, nvpc - 1) * nq];
            const int* qn = &L.Q.cell_nodes[(size_t)e * nq];
            for (int l = 0; l < nq; ++l)
                if (ok[l]) out.push_back(qn[l]);
        }
        sort_unique_tail(out, s1);
        NV[v] = (int)(s1 - s0);
        NP[v] = (int)(out.size() - s1);
    }, 192, 4);
    pc.lap("star lists");
    // vertices with a non-empty patch, in order; patch p lists d blocks of its
    // velocity nodes (one per component), then its pressures
    std::vector<int> vid;
    vid.reserve(m.nv);
    for (int v = 0; v < m.nv; ++v)
        if (NV[v] + NP[v] > 0) vid.push_back(v);
    const int np = (int)vid.size();
    std::vector<int> sz(np);
    for (int p = 0; p < np; ++p) sz[p] = d * NV[vid[p]] + NP[vid[p]];
    L.patch_off.resize(np + 1);
    parallel_scan(sz.data(), np, L.patch_off.data());
    L.patch_dofs.resize(L.patch_off[np]);
    L.patch_nv.resize(np);
    parallel_for(np, [&](int lo, int hi, int) {
        for (int p = lo; p < hi; ++p) {
            const int v = vid[p];
            const int* src = lists.begin(v);
            int* dst = L.patch_dofs.data() + L.patch_off[p];
            const int nvv = NV[v];
            for (int c = 0; c < d; ++c)
                for (int x = 0; x < nvv; ++x) *dst++ = c * L.nVf + src[x];
            for (int x = 0; x < NP[v]; ++x) *dst++ = d * L.nVf + src[nvv + x];
            L.patch_nv[p] = nvv;
        }
    }, 128, 4);
    pc.lap("patch dofs");
}

// Finite-element interpolation (Sec. 3.1): the coarse basis evaluated at the
// fine nodes, each fine node located in the coarse cell that contains the
// fine cell owning it.  Entries with |v| <= 1e-14 (exact lattice zeros) are
// dropped.
static CSR scalar_interp(const Mesh& mf, const Space& Vf, const Mesh& mc, const Space& Vc,
                         const RefElement& rec, const std::vector<int>* parent, const RefElement* ref_f) {
    const int d = mf.d, nbc = Vc.nb;
    CSR P;
    P.nr = Vf.n;
    P.ncol = Vc.n;
    // On one mesh (a p-transfer) a fine node with local index l sits at the
    // reference point alpha_l / k_f of its owner cell, the coarse cell too:
    // the coarse basis values there are one table row per l.
    std::vector<double> tab;
    if (!parent && ref_f && ref_f->k > 0 && ref_f->nb == Vf.nb) {
        tab.resize((size_t)ref_f->nb * nbc);
        for (int l = 0; l < ref_f->nb; ++l) {
            double xi[3] = {0, 0, 0};
            for (int a = 0; a < d; ++a) xi[a] = (double)ref_f->alpha[l][a + 1] / ref_f->k;
            rec.eval(xi, tab.data() + (size_t)l * nbc);
        }
    }
    // a row has at most nbc entries: fill fixed slots in parallel, then compact
    std::vector<int> cnt(Vf.n);
    fvec<int> scol((size_t)Vf.n * nbc);
    fvec<double> sval((size_t)Vf.n * nbc);
    parallel_for(Vf.n, [&](int lo, int hi, int) {
        double vbuf[320];
        std::pair<int, double> row[320];
        for (int i = lo; i < hi; ++i) {
            int fc = Vf.owner_cell[i];
            int cc = parent ? (*parent)[fc] : fc;
            const double* val = vbuf;
            if (!tab.empty()) {
                val = tab.data() + (size_t)Vf.owner_local[i] * nbc;
            } else {
                CellGeom g = cell_geom(mc, cc);
                const int* cv = &mc.C[(size_t)cc * (d + 1)];
                double xi[3] = {0, 0, 0};
                for (int a = 0; a < d; ++a) {
                    double s = 0;
                    for (int c = 0; c < d; ++c) s += g.Jinv[a * d + c] * (Vf.X[(size_t)i * d + c] - mc.X[(size_t)cv[0] * d + c]);
                    xi[a] = s;
                }
                rec.eval(xi, vbuf);
            }
            int m = 0;
            for (int l = 0; l < nbc; ++l)
                if (std::fabs(val[l]) > 1e-14) row[m++] = {Vc.cell_nodes[(size_t)cc * nbc + l], val[l]};
            std::sort(row, row + m);
            cnt[i] = m;
            for (int t = 0; t < m; ++t) {
                scol[(size_t)i * nbc + t] = row[t].first;
                sval[(size_t)i * nbc + t] = row[t].second;
            }
        }
    });
    P.rp.assign(P.nr + 1, 0);
    {
        long long sp = 0;
        for (int i = 0; i < P.nr; ++i) P.rp[i + 1] = index_total(sp += cnt[i], "transfer");
    }
    P.ci.resize(P.rp[P.nr]);
    P.v.resize(P.rp[P.nr]);
    parallel_for(P.nr, [&](int lo, int hi, int) {
        for (int i = lo; i < hi; ++i)
            for (int t = 0; t < cnt[i]; ++t) {
                P.ci[P.rp[i] + t] = scol[(size_t)i * nbc + t];
                P.v[P.rp[i] + t] = sval[(size_t)i * nbc + t];
            }
    });
    return P;
}

static void monolithic_interp(const Mesh& mf, Level& F, const Mesh& mc, const Level& C,
                              const RefElement& recV, const RefElement& recQ, const std::vector<int>* parent,
                              const RefElement* refV_f, const RefElement* refQ_f) {
    CSR PV = scalar_interp(mf, F.V, mc, C.V, recV, parent, refV_f);
    CSR PQ = scalar_interp(mf, F.Q, mc, C.Q, recQ, parent, refQ_f);
    const int d = mf.d;
    CSR& P = F.P;
    P.nr = F.n_free;
    P.ncol = C.n_free;
    std::vector<int> vrow(F.nVf);
    for (int i = 0; i < F.V.n; ++i)
        if (F.vfree[i] >= 0) vrow[F.vfree[i]] = i;
    // free coarse columns only; the coarse free numbering follows node order,
    // so rows of PV (sorted by coarse node) stay sorted
    std::vector<int> vcount(F.nVf);
    parallel_for(F.nVf, [&](int lo, int hi, int) {
        for (int f = lo; f < hi; ++f) {
            int i = vrow[f], c = 0;
            for (int p = PV.rp[i]; p < PV.rp[i + 1]; ++p) c += C.vfree[PV.ci[p]] >= 0;
            vcount[f] = c;
        }
    });
    P.rp.assign(P.nr + 1, 0);
    for (int c = 0; c < d; ++c)
        for (int f = 0; f < F.nVf; ++f) P.rp[c * F.nVf + f + 1] = vcount[f];
    for (int q = 0; q < F.Q.n; ++q) P.rp[d * F.nVf + q + 1] = PQ.rp[q + 1] - PQ.rp[q];
    {
        long long sp = 0;
        for (int r = 0; r < P.nr; ++r) P.rp[r + 1] = index_total(sp += P.rp[r + 1], "transfer");
    }
    P.ci.resize(P.rp[P.nr]);
    P.v.resize(P.rp[P.nr]);
    parallel_for(F.nVf, [&](int lo, int hi, int) {
        for (int f = lo; f < hi; ++f) {
            int i = vrow[f];
            for (int c = 0; c < d; ++c) {
                int o = P.rp[c * F.nVf + f];
                for (int p = PV.rp[i]; p < PV.rp[i + 1]; ++p) {
                    int jc = C.vfree[PV.ci[p]];
                    if (jc < 0) continue;
                    P.ci[o] = c * C.nVf + jc;
                    P.v[o++] = PV.v[p];
                }
            }
        }
    });
    parallel_for(F.Q.n, [&](int lo, int hi, int) {
        for (int q = lo; q < hi; ++q) {
            int o = P.rp[d * F.nVf + q];
            for (int p = PQ.rp[q]; p < PQ.rp[q + 1]; ++p) {
                P.ci[o] = d * C.nVf + PQ.ci[p];
                P.v[o++] = PQ.v[p];
            }
        }
    });
    F.R = transpose(P);
}

const RefElement& reference_element(int d, int k) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, RefElement> refs;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(d, k);
    auto it = refs.find(key);
    if (it == refs.end()) { refs[key].init(d, k); it = refs.find(key); }
    return it->second;
}

void build_hierarchy(const Mesh& coarse, const HierarchySpec& spec, const double* nu_cell, Hierarchy& H,
                     const std::function<void(int, int)>& on_level) {
    double t0 = now_ms();
    const int d = coarse.d;
    if (d != 2 && d != 3) throw std::invalid_argument("dim must be 2 or 3");
    if (spec.schedule.empty()) throw std::invalid_argument("empty p-schedule");
    for (int x : coarse.C)
        if (x < 0 || x >= coarse.nv) throw std::invalid_argument("cell vertex index out of range");
    std::vector<Mesh> fine_to_coarse{coarse};
    std::vector<std::vector<int>> par;
    for (int r = 0; r < spec.n_refine; ++r) {
        std::vector<int> p;
        fine_to_coarse.push_back(refine_uniform(fine_to_coarse.back(), p));
        par.push_back(std::move(p));
    }
    if (spec.barycentric) {
        std::vector<int> p;
        fine_to_coarse.push_back(refine_alfeld(fine_to_coarse.back(), p));
        par.push_back(std::move(p));
    }
    H.meshes.assign(fine_to_coarse.rbegin(), fine_to_coarse.rend());
    H.parents.assign(par.rbegin(), par.rend());
    const int nm = (int)H.meshes.size();
    for (int e = 0; e < H.meshes.back().nc; ++e) {
        // reject degenerate coarse cells
        CellGeom g = cell_geom(H.meshes.back(), e);
        if (!(g.detabs > 0) || !std::isfinite(g.detabs)) throw std::invalid_argument("degenerate coarse cell");
    }
    // viscosity per cell on every mesh (coarse cell = mean of its children)
    std::vector<std::vector<double>> nus(nm);
    if (nu_cell) {
        nus[0].assign(nu_cell, nu_cell + H.meshes[0].nc);
        for (int i = 0; i + 1 < nm; ++i) {
            std::vector<double> s(H.meshes[i + 1].nc, 0.0), c(H.meshes[i + 1].nc, 0.0);
            for (int e = 0; e < H.meshes[i].nc; ++e) { s[H.parents[i][e]] += nus[i][e]; c[H.parents[i][e]] += 1; }
            for (size_t e = 0; e < s.size(); ++e) s[e] /= c[e];
            nus[i + 1] = s;
        }
    }
    // topologies on demand: the coarsest mesh's now, the others when their
    // first level is built (so that a coarsest-first build starts at once)
    std::vector<Topology> topo(nm);
    std::vector<char> have_topo(nm, 0);
    auto need_topo = [&](int i) {
        if (!have_topo[i]) { build_topology(H.meshes[i], topo[i]); have_topo[i] = 1; }
    };
    need_topo(nm - 1);
    double t1 = now_ms();
    H.t_mesh_ms = t1 - t0;
    // levels: p-levels on the finest mesh, then the hMG degree on every mesh
    struct LS { int mesh, family, k; bool p; };
    std::vector<LS> ls;
    const int np = (int)spec.schedule.size() - 1;
    for (int i = 0; i < np; ++i) ls.push_back({0, i == 0 ? spec.family : 0, spec.schedule[i], true});
    const int q = spec.schedule.back();
    for (int mi = 0; mi < nm; ++mi) ls.push_back({mi, (np == 0 && mi == 0) ? spec.family : 0, q, false});
    if ((int)ls.size() > 16) throw std::invalid_argument("too many levels");
    H.levels.assign(ls.size(), Level());
    // reference elements and tensors depend on (d, k) only: computed once per
    // process and kept (std::map entries do not move on insertion)
    static std::mutex ref_mu;
    static std::map<std::pair<int, int>, RefTensors> tensors;
    auto ref = [&](int dd, int kk) -> const RefElement& { return reference_element(dd, kk); };
    // one level: spaces, operator data (or host matrices), callback stage 0,
    // patches, callback stage 1; the phase times merge under tmu
    std::mutex tmu;
    auto build_one = [&](size_t l) {
        Level& L = H.levels[l];
        L.d = d;
        L.family = ls[l].family;
        L.k = ls[l].k;
        L.mesh_index = ls[l].mesh;
        L.p_level = ls[l].p;
        if (L.k < 2 || L.k > 10) throw std::invalid_argument("velocity degree must be in [2, 10]");
        if (L.family == 1 && L.k < d) throw std::invalid_argument("Scott-Vogelius needs k >= dim");
        const Mesh& m = H.meshes[L.mesh_index];
        double ta = now_ms();
        need_topo(L.mesh_index);
        L.max_cells = topo[L.mesh_index].max_valence;
        const RefElement& rv = ref(d, L.k);
        const RefElement& rq = ref(d, L.k - 1);
        build_space(m, topo[L.mesh_index], rv, true, L.V);
        build_space(m, topo[L.mesh_index], rq, L.family == 0, L.Q);
        const RefTensors* rtp;
        {
            std::lock_guard<std::mutex> g(ref_mu);
            auto rkey = std::make_pair(d * 100 + L.k, 0);
            auto rit = tensors.find(rkey);
            if (rit == tensors.end()) { tensors[rkey].init(rv, rq); rit = tensors.find(rkey); }
            rtp = &rit->second;
        }
        const RefTensors& RT = *rtp;
        double tb = now_ms();
        L.RT = RT;
        L.nu_cells = nus[L.mesh_index];
        L.host_matrices = spec.device_assembly_finest_only ? l != 0 : (!spec.device_assembly || l + 1 == ls.size());
        if (L.host_matrices) assemble_level(m, L, RT, nus[L.mesh_index], l == 0);
        else prepare_level(m, L, RT);
        double tc = now_ms();
        double t_cb = 0;
        if (on_level) {
            on_level((int)l, 0);
            const double tcb = now_ms();
            t_cb += tcb - tc;
            tc = tcb;
        }
        if (l + 1 < ls.size() && !spec.skip_patches) build_patches(m, topo[L.mesh_index], L);
        const double td = now_ms();
        if (host_trace())
            std::fprintf(stderr, "[sfem] level %zu: spaces %.3f  operator data %.3f  patches %.3f ms\n", l, tb - ta,
                         tc - tb, td - tc);
        if (on_level) {
            on_level((int)l, 1);
            t_cb += now_ms() - td;
        }
        std::lock_guard<std::mutex> g(tmu);
        H.t_spaces_ms += tb - ta;
        H.t_matrices_ms += tc - tb;
        H.t_patches_ms += td - tc;
        H.t_callbacks_ms += t_cb;
    };
    std::vector<size_t> order;
    const bool side = spec.coarsest_first && spec.coarsest_thread && ls.size() > 1;
    if (spec.coarsest_first && !side) order.push_back(ls.size() - 1);
    for (size_t l = 0; l + 1 < ls.size(); ++l) order.push_back(l);
    if (!spec.coarsest_first) order.push_back(ls.size() - 1);
    {
        // the coarsest level beside the others (joined before this scope
        // ends, also when a level throws)
        std::exception_ptr side_err;
        std::thread th;
        if (side)
            th = std::thread([&] {
                t_pool_inline = true;
                try {
                    build_one(ls.size() - 1);
                } catch (...) {
                    side_err = std::current_exception();
                }
            });
        struct Join {
            std::thread& t;
            ~Join() {
                if (t.joinable()) t.join();
            }
        } join{th};
        for (size_t l : order) build_one(l);
        if (th.joinable()) th.join();
        if (side_err) std::rethrow_exception(side_err);
    }
    double tt = now_ms();
    for (size_t l = 0; l + 1 < ls.size() && !spec.device_transfers; ++l) {
        Level &F = H.levels[l], &C = H.levels[l + 1];
        const std::vector<int>* par_map = (F.mesh_index == C.mesh_index) ? nullptr : &H.parents[F.mesh_index];
        monolithic_interp(H.meshes[F.mesh_index], F, H.meshes[C.mesh_index], C, ref(d, C.k), ref(d, C.k - 1), par_map,
                          &ref(d, F.k), &ref(d, F.k - 1));
    }
    H.t_transfers_ms = now_ms() - tt;
    H.t_assembly_ms = now_ms() - t1 - H.t_callbacks_ms;
}

// rows [0, nr) and columns [0, nc) of a CSR (the column order of each row kept)
static CSR csr_leading_block(const CSR& a, int nr, int nc) {
    CSR b;
    b.nr = nr;
    b.ncol = nc;
    b.rp.assign(nr + 1, 0);
    parallel_for(nr, [&](int lo, int hi, int) {
        for (int r = lo; r < hi; ++r) {
            int cnt = 0;
            for (int p = a.rp[r]; p < a.rp[r + 1]; ++p) cnt += a.ci[p] < nc;
            b.rp[r + 1] = cnt;
        }
    });
    for (int r = 0; r < nr; ++r) b.rp[r + 1] += b.rp[r];
    b.ci.resize(b.rp[nr]);
    b.v.resize(b.rp[nr]);
    parallel_for(nr, [&](int lo, int hi, int) {
        for (int r = lo; r < hi; ++r) {
            int o = b.rp[r];
            for (int p = a.rp[r]; p < a.rp[r + 1]; ++p)
                if (a.ci[p] < nc) { b.ci[o] = a.ci[p]; b.v[o] = a.v[p]; ++o; }
        }
    });
    return b;
}

void velocity_hierarchy(Hierarchy& S, Hierarchy& A) {
    A.meshes = S.meshes;
    A.parents = S.parents;
    A.levels.assign(S.levels.size(), Level());
    for (size_t l = 0; l < S.levels.size(); ++l) {
        const Level& F = S.levels[l];
        Level& L = A.levels[l];
        if (F.host_matrices && F.K.rp.empty()) throw std::runtime_error("velocity_hierarchy: level without operator");
        L.d = F.d;
        L.family = 0;
        L.k = F.k;
        L.mesh_index = F.mesh_index;
        L.p_level = F.p_level;
        L.V = F.V;
        L.vfree = F.vfree;
        L.nVf = F.nVf;
        L.nQ = 0;
        L.n_free = F.nVf;
        if (F.host_matrices) L.K = csr_leading_block(F.K, F.nVf, F.nVf);
        L.RT = F.RT;
        L.nu_cells = F.nu_cells;
        L.host_matrices = F.host_matrices;
        if (l + 1 < S.levels.size()) {
            L.P = csr_leading_block(F.P, F.nVf, S.levels[l + 1].nVf);
            L.R = transpose(L.P);
            // ASMStarPC: the free nodes whose owning entity contains vertex v
            const int nv = S.meshes[F.mesh_index].nv;
            std::vector<std::vector<int>> star(nv);
            for (int i = 0; i < F.V.n; ++i) {
                const int f = F.vfree[i];
                if (f < 0) continue;
                for (int v : F.V.support[i])
                    if (v >= 0) star[v].push_back(f);
            }
            L.patch_off.assign(1, 0);
            for (int v = 0; v < nv; ++v) {
                if (star[v].empty()) continue;
                std::sort(star[v].begin(), star[v].end());
                L.patch_dofs.insert(L.patch_dofs.end(), star[v].begin(), star[v].end());
                L.patch_off.push_back((int)L.patch_dofs.size());
                L.patch_nv.push_back(0);      // no velocity/pressure structure: Gauss-Jordan inverses
            }
        }
    }
}

std::vector<double> reference_mass(int d, int k) {
    RefElement e;
    e.init(d, k);
    RefTensors t;
    t.init(e, e);
    return t.M;
}

}  // namespace sfem
