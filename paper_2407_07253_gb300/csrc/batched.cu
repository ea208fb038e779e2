// Kernels of the batched V-cycle; see batched.cuh.
#include "batched.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

namespace sbat {

namespace {

inline int grid_of(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

__global__ void k_to_interleaved(int n, int nrhs, int m, const double* __restrict__ r, float* __restrict__ X) {
    const long long total = (long long)n * m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / m), c = (int)(t - (long long)j * m);
        X[t] = c < nrhs ? (float)r[(long long)c * n + j] : 0.0f;
    }
}

__global__ void k_from_interleaved(int n, int nrhs, int m, const float* __restrict__ X, double* __restrict__ z) {
    const long long total = (long long)n * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n), j = (int)(t - (long long)c * n);
        z[t] = (double)X[(long long)j * m + c];
    }
}

// A group of m/2 lanes per row, one float2 of right-hand sides per lane;
// the row's entries are walked four at a time with their loads issued
// together.
template <int MODE>
__global__ void __launch_bounds__(256) k_spmm(int nr, int m, const int* __restrict__ rp, const int* __restrict__ ci,
                                              const float* __restrict__ av, const float2* __restrict__ X,
                                              float2* __restrict__ Y, const float2* __restrict__ B) {
    const int L = m >> 1;                                   // lanes per row
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int row = (int)(gt / L), c2 = (int)(gt - (long long)row * L);
    if (row >= nr) return;
    const int s = __ldg(rp + row), e = __ldg(rp + row + 1);
    float2 acc = make_float2(0.f, 0.f);
    int p = s;
    for (; p + 4 <= e; p += 4) {
        int c[4];
        float a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { c[u] = __ldg(ci + p + u); a[u] = __ldg(av + p + u); }
        float2 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldg(X + (long long)c[u] * L + c2);
#pragma unroll
        for (int u = 0; u < 4; ++u) { acc.x = fmaf(a[u], x[u].x, acc.x); acc.y = fmaf(a[u], x[u].y, acc.y); }
    }
    for (; p < e; ++p) {
        const float a = __ldg(av + p);
        const float2 x = __ldg(X + (long long)__ldg(ci + p) * L + c2);
        acc.x = fmaf(a, x.x, acc.x);
        acc.y = fmaf(a, x.y, acc.y);
    }
    const long long o = (long long)row * L + c2;
    if (MODE == 0) Y[o] = acc;
    else if (MODE == 1) { float2 y = Y[o]; y.x += acc.x; y.y += acc.y; Y[o] = y; }
    else { const float2 b = B[o]; Y[o] = make_float2(b.x - acc.x, b.y - acc.y); }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros
// and reads nothing
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

constexpr int KC = 16;          // columns of K_p^{-1} per ring slot (two k-steps)
constexpr int MIN_STAGES = 4;   // ring slots per warp: 4, 6 or 8, the most that fit
constexpr int SLOT = 16 * KC;   // floats per slot: 16 rows x KC columns

// row stride (floats) of the transposed block R_p^T in shared memory: at
// least n rounded up to 16, and 16 mod 32, so that the quarter-warps of a
// 128-bit fragment load cover all 32 banks once
__host__ __device__ inline int rt_ld(int n) {
    const int n16 = (n + 15) & ~15;
    return (n16 & 31) == 16 ? n16 : n16 + 16;
}

// One CTA of NW warps per patch (NW set by the launch, <= 16).
//
// R_p^T (m x n, zero-padded to a multiple of 16 columns) is gathered into
// shared memory once, already rounded to TF32 in the TF32 mode.  Warp w
// computes the 16-row blocks w, w + NW, ... of Y_p = K_p^{-1} R_p.  For each
// it streams its 16 rows of K_p^{-1} from HBM through a private ring of
// ST slots of KC columns (cp.async, ST - 1 slots in flight, every
// entry read once).  K_p^{-1} is symmetric, so row i of the block is column
// i of the column-major inverse: each slot row is 64 contiguous bytes.
//
// The k index inside each 16-column slot is permuted so that one 128-bit
// shared load gives a lane its operands for two k-steps: for the m16n8k8
// TF32 fragments (g = lane / 4, t = lane % 4)
//   A (16 x 8, row): a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (8 x 8, col):  b0 (t, g), b1 (t + 4, g)
//   D (16 x 8):      d0 (g, 2t), d1 (g, 2t + 1), d2 (g + 8, 2t), d3 (g + 8, 2t + 1)
// the fragment k indices t and t + 4 of the first k-step stand for slot
// columns 4t and 4t + 1, those of the second for 4t + 2 and 4t + 3.  A and B
// use the same map, so the products pair up exactly.
template <int M, int MODE, int ST>
__global__ void __launch_bounds__(512, 1) k_patch_gemm(int npatch, const int* __restrict__ plist,
                                                    const int* __restrict__ poff,
                                                    const int* __restrict__ pdofs, const long long* __restrict__ ioff,
                                                    const float* __restrict__ inv, const float* __restrict__ X,
                                                    const float* __restrict__ wt, float* __restrict__ Yb) {
    extern __shared__ __align__(128) float smem_pg[];
    constexpr int NT = M / 8, Q = M / 4;
    const int p = plist ? __ldg(plist + blockIdx.x) : (int)blockIdx.x;     // one CTA per listed patch
    const int s = poff[p], n = poff[p + 1] - s;
    const int n16 = (n + 15) & ~15, ld = (n + 3) & ~3, ldk = rt_ld(n);
    const int nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    float* Rt = smem_pg;                                     // [M][ldk]
    float* ring = smem_pg + M * ldk + warp * (ST * SLOT);
    const uint32_t ring_s = smem_u32(ring);
    const float* A = inv + ioff[p];

    // this warp's work items: (row block, slot), row blocks warp, warp + nw,
    // ...; slots of KC columns 0 .. ng - 1
    const int nrb = (n + 15) >> 4, ng = n16 / KC;
    const int items = warp < nrb ? ((nrb - 1 - warp) / nw + 1) * ng : 0;
    int is_rb = warp, is_g = 0, is_it = 0;                   // next item to issue
    auto issue = [&]() {
        if (is_it < items) {
            const uint32_t slot = ring_s + 4u * (uint32_t)((is_it % ST) * SLOT);
            const int c0 = is_g * KC;
#pragma unroll
            for (int q = lane; q < 16 * (KC / 4); q += 32) {
                const int rl = q / (KC / 4), j = q % (KC / 4), r = is_rb * 16 + rl, c = c0 + 4 * j;
                const bool ok = r < n && c < ld;
                const float* src = ok ? A + (long long)r * ld + c : A;
                cp_async16(slot + 4u * (uint32_t)(rl * KC + 4 * j), src, ok ? 16 : 0);
            }
            if (++is_g == ng) { is_g = 0; is_rb += nw; }
        }
        ++is_it;
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < ST - 1; ++i) issue();

    // R_p^T -> shared while the first slots are in flight: tpr threads per
    // DoF row, each loading 16-byte pieces of the row four at a time
    {
        const int tpr = blockDim.x >= n16 ? blockDim.x / n16 : 1;
        const int rows_per_pass = blockDim.x / tpr;
        const int jt = threadIdx.x % tpr;
        for (int k = threadIdx.x / tpr; k < n16 && threadIdx.x < tpr * rows_per_pass; k += rows_per_pass) {
            const float4* xr = k < n ? reinterpret_cast<const float4*>(X + (long long)__ldg(pdofs + s + k) * M) : nullptr;
            for (int j0 = jt; j0 < Q; j0 += 4 * tpr) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u * tpr;
                    v[u] = (xr && j < Q) ? __ldg(xr + j) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = j0 + u * tpr;
                    if (j < Q) {
                        if (MODE == GEMM_TF32) {
                            v[u].x = __uint_as_float(to_tf32(v[u].x));
                            v[u].y = __uint_as_float(to_tf32(v[u].y));
                            v[u].z = __uint_as_float(to_tf32(v[u].z));
                            v[u].w = __uint_as_float(to_tf32(v[u].w));
                        }
                        float* dst = Rt + (4 * j) * ldk + k;
                        dst[0] = v[u].x;
                        dst[ldk] = v[u].y;
                        dst[2 * ldk] = v[u].z;
                        dst[3 * ldk] = v[u].w;
                    }
                }
            }
        }
    }
    __syncthreads();

    float d[NT][4], w0 = 0.f, w1 = 0.f;
    int rb = warp, gi = 0;
    for (int it = 0; it < items; ++it) {
        if (gi == 0) {
#pragma unroll
            for (int q = 0; q < NT; ++q) d[q][0] = d[q][1] = d[q][2] = d[q][3] = 0.f;
            const int r0 = rb * 16 + g, r1 = r0 + 8;     // weights, needed at the end of the row block
            w0 = r0 < n ? __ldg(wt + __ldg(pdofs + s + r0)) : 0.f;
            w1 = r1 < n ? __ldg(wt + __ldg(pdofs + s + r1)) : 0.f;
        }
        issue();
        cp_async_wait<ST - 1>();
        __syncwarp();
        const float* sl = ring + (it % ST) * SLOT;
        const float4 A0 = *reinterpret_cast<const float4*>(sl + g * KC + 4 * t);
        const float4 A1 = *reinterpret_cast<const float4*>(sl + (g + 8) * KC + 4 * t);
        __syncwarp();            // the next iteration refills this slot
        const float av[2][4] = {{A0.x, A1.x, A0.y, A1.y}, {A0.z, A1.z, A0.w, A1.w}};
        uint32_t ah[2][4], al[2][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                ah[u][x] = to_tf32(av[u][x]);
                al[u][x] = __float_as_uint(av[u][x] - __uint_as_float(ah[u][x]));
            }
        const float* bp = Rt + g * ldk + gi * KC + 4 * t;
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const float4 bv = *reinterpret_cast<const float4*>(bp + q * 8 * ldk);
            const float b[2][2] = {{bv.x, bv.y}, {bv.z, bv.w}};
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (MODE == GEMM_3XTF32) {
                    const uint32_t bh0 = to_tf32(b[u][0]), bh1 = to_tf32(b[u][1]);
                    const uint32_t bl0 = __float_as_uint(b[u][0] - __uint_as_float(bh0));
                    const uint32_t bl1 = __float_as_uint(b[u][1] - __uint_as_float(bh1));
                    mma_tf32(d[q], al[u], bh0, bh1);
                    mma_tf32(d[q], ah[u], bl0, bl1);
                    mma_tf32(d[q], ah[u], bh0, bh1);
                } else {
                    mma_tf32(d[q], ah[u], __float_as_uint(b[u][0]), __float_as_uint(b[u][1]));
                }
            }
        }
        if (++gi == ng) {
            const int r0 = rb * 16 + g, r1 = r0 + 8;
#pragma unroll
            for (int q = 0; q < NT; ++q) {
                const int c = q * 8 + 2 * t;
                if (r0 < n)
                    *reinterpret_cast<float2*>(Yb + (long long)(s + r0) * M + c) = make_float2(w0 * d[q][0], w0 * d[q][1]);
                if (r1 < n)
                    *reinterpret_cast<float2*>(Yb + (long long)(s + r1) * M + c) = make_float2(w1 * d[q][2], w1 * d[q][3]);
            }
            gi = 0;
            rb += nw;
        }
    }
    cp_async_wait<0>();
}

// ---- TF32 mode on the 5th-generation tensor cores (tcgen05) -------------
//
// A persistent kernel (one CTA per SM) walks its share of the patches with a
// warp-specialised pipeline over stages of KS = 16 inverse columns:
//   warp 0, lane 0   TMA: the stage's rows of K_p^{-1} (one 128-row box per
//                    row tile, 64-byte swizzle, zero fill outside the patch)
//                    through the per-patch tensor map.  K_p^{-1} is
//                    symmetric, so row r of the product's left factor is the
//                    stored column r: each box row is 64 contiguous bytes.
//   warps 2-9        the stage's 16 rows of R_p, gathered from X, rounded to
//                    TF32 and written as the K-major B operand (8 x 16-byte
//                    core matrices, no swizzle), then fenced to the async
//                    proxy; each warp takes every G-th stage, so up to
//                    G = min(8, stages) gathers are in flight.
//   warp 1, lane 0   waits for both, issues the stage's M = 128, N = np,
//                    K = 8 MMAs (one per row tile and k-step) into the
//                    patch's tensor-memory accumulator and commits them to
//                    the stage's empty barrier; after the patch's last stage
//                    it commits the accumulator to the epilogue.
//   warps 10-13      epilogue: tensor memory -> registers (the 32 lanes of
//                    warp w % 4), times the partition-of-unity weight, -> Yb.
// Two accumulators alternate between patches when they fit in the 512
// tensor-memory columns, so the epilogue of one patch overlaps the MMAs of
// the next.  All mbarrier waits are bounded; on a timeout the CTA records it
// in *status, stops every role and returns.
namespace tc {

constexpr int KS = 16;                    // inverse columns per stage: two K = 8 steps
constexpr int A_TILE = 128 * KS * 4;      // bytes of one 128-row tile of a stage (8 KB)
constexpr int B_GROUP = (KS / 4) * 128;   // bytes between 8-row groups of the B operand
constexpr int HDR = 1024;                 // barriers, tensor-memory address, abort flag
constexpr int GATHER_WARPS = 8;           // stages gathered concurrently
constexpr int THREADS = 32 * (2 + GATHER_WARPS + 4);
constexpr long long WAIT_LIMIT = 1ll << 22;

__host__ __device__ constexpr int np_of(int m) { return m < 16 ? 16 : m; }
__host__ __device__ inline int tiles_of(int n) { return (n + 127) >> 7; }
// a stage: the inverse's 128-row tiles (split: the hi tiles, then the lo
// tiles), then the B operand (split: its hi part, then its lo part)
__host__ __device__ inline int stage_bytes(int maxn, int np, bool split = false) {
    const int f = split ? 2 : 1;
    return (f * tiles_of(maxn) * A_TILE + f * np * KS * 4 + 1023) & ~1023;
}
__host__ __device__ inline int acc_cols(int maxn, int np) { return tiles_of(maxn) * np; }
__host__ __device__ inline int acc_bufs(int maxn, int np) { return 2 * acc_cols(maxn, np) <= 512 ? 2 : 1; }
__host__ __device__ inline int tmem_cols(int maxn, int np) {
    int need = acc_bufs(maxn, np) * acc_cols(maxn, np), c = 32;
    while (c < need) c <<= 1;
    return c;
}

// shared-memory matrix descriptors (K-major): without swizzle (8-row x
// 16-byte core matrices, lbo along K, sbo along M / N) and with the 64-byte
// swizzle of the TMA boxes (8-row atoms of 64-byte rows, sbo = 512)
__device__ __forceinline__ uint64_t desc_plain(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
__device__ __forceinline__ uint64_t desc_sw64(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) |
           (4ull << 61);
}

// instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = np
__host__ __device__ constexpr uint32_t idesc(int np) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(np >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait; false (and the CTA's abort flag set) after `limit` polls,
// or at once if another role has already given up
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, volatile int* abort_flag,
                                          long long limit = WAIT_LIMIT) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try(a, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// self-test of the bounded wait: one CTA waits on an mbarrier that nothing
// arrives on; *result = 2 when the wait gives up after `limit` polls and the
// kernel returns (1 would mean the phase completed)
__global__ void k_wait_probe(long long limit, int* result) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    const uint32_t a = smem_u32(&bar);
    if (threadIdx.x == 0) {
        mbar_init(a, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(a, 0, &abort_flag, limit);
    __syncthreads();
    if (threadIdx.x == 0) *result = ok ? 1 : 2;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, uint32_t mbar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(tmap), "r"(mbar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

// SPLIT (3xTF32): the inverse comes as two arrays, hi = TF32(a) and
// lo = a - hi (tmaps over hi, tmaps_lo over lo), R as hi = TF32(r) and
// lo = TF32(r - hi), and every k-step issues three MMAs into the same
// accumulator: lo x hi, hi x lo, hi x hi (lo x lo, of relative size 2^-22,
// is dropped).  This keeps FP32 accuracy on the tensor cores.
template <int M, int ST, bool SPLIT>
__global__ void __launch_bounds__(THREADS, 1) k_patch_gemm_tc(int npatch, int maxn, const int* __restrict__ plist,
                                                              const int* __restrict__ poff,
                                                              const int* __restrict__ pdofs,
                                                              const CUtensorMap* __restrict__ tmaps,
                                                              const CUtensorMap* __restrict__ tmaps_lo,
                                                              const float* __restrict__ X,
                                                              const float* __restrict__ wt, float* __restrict__ Yb,
                                                              int* status) {
    constexpr int NP = np_of(M);
    constexpr int F = SPLIT ? 2 : 1;
    extern __shared__ __align__(1024) unsigned char smem_tc[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t base = smem_u32(smem_tc);
    const uint32_t full0 = base, empty0 = base + 8 * ST, accf0 = base + 16 * ST, acce0 = accf0 + 16;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_tc + 16 * ST + 32);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem_tc + 16 * ST + 36);
    const int sbytes = stage_bytes(maxn, NP, SPLIT);
    const uint32_t stage0 = (base + HDR + 1023) & ~1023u;     // swizzle atoms need 1024-byte alignment
    const uint32_t lo_off = (uint32_t)(tiles_of(maxn) * A_TILE);     // lo tiles inside a stage (SPLIT)
    const uint32_t b_off = (uint32_t)(F * tiles_of(maxn) * A_TILE);  // B operand inside a stage
    constexpr uint32_t BLO = (uint32_t)(NP * KS * 4);                 // its lo part after the hi part (SPLIT)
    const int nbuf = acc_bufs(maxn, NP), ccols = acc_cols(maxn, NP), ncols = tmem_cols(maxn, NP);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(full0 + 8 * s, 1 + 32);      // TMA arrival with the byte count + one gather warp
            mbar_init(empty0 + 8 * s, 1);          // MMA commit
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);           // MMA commit of a patch's last stage
            mbar_init(acce0 + 8 * b, 128);         // epilogue threads
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA ---
        if (lane == 0) {
            int it = 0;
            for (int i = blockIdx.x; i < npatch; i += gridDim.x) {
                const int p = plist ? __ldg(plist + i) : i;
                const int n = poff[p + 1] - poff[p], tiles = tiles_of(n), nst = (n + KS - 1) / KS;
                const CUtensorMap* tm = tmaps + p;
                const CUtensorMap* tml = SPLIT ? tmaps_lo + p : nullptr;
                for (int j = 0; j < nst; ++j, ++it) {
                    const int s = it % ST;
                    if (it >= ST && !mbar_wait(empty0 + 8 * s, ((it / ST) - 1) & 1, abort_flag)) goto done;
                    const uint32_t st = stage0 + (uint32_t)(s * sbytes);
                    mbar_expect_tx(full0 + 8 * s, (uint32_t)(F * tiles * A_TILE));
                    for (int mt = 0; mt < tiles; ++mt) {
                        tma_load_2d(st + mt * A_TILE, tm, full0 + 8 * s, j * KS, mt * 128);
                        if (SPLIT) tma_load_2d(st + lo_off + mt * A_TILE, tml, full0 + 8 * s, j * KS, mt * 128);
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA ---
        if (lane == 0) {
            constexpr uint32_t ID = idesc(NP);
            int it = 0, pc = 0;
            for (int i = blockIdx.x; i < npatch; i += gridDim.x, ++pc) {
                const int p = plist ? __ldg(plist + i) : i;
                const int n = poff[p + 1] - poff[p], tiles = tiles_of(n), nst = (n + KS - 1) / KS;
                const int b = pc % nbuf;
                if (pc >= nbuf && !mbar_wait(acce0 + 8 * b, ((pc / nbuf) - 1) & 1, abort_flag)) goto done;
                fence_after();
                const uint32_t acc = tmem + (uint32_t)(b * ccols);
                for (int j = 0; j < nst; ++j, ++it) {
                    const int s = it % ST;
                    if (!mbar_wait(full0 + 8 * s, (it / ST) & 1, abort_flag)) goto done;
                    fence_after();
                    const uint32_t st = stage0 + (uint32_t)(s * sbytes);
#pragma unroll
                    for (int u = 0; u < KS / 8; ++u) {
                        const uint64_t bd = desc_plain(st + b_off + (uint32_t)(u * 2 * 128), 128, B_GROUP);
                        for (int mt = 0; mt < tiles; ++mt) {
                            const uint64_t ad = desc_sw64(st + (uint32_t)(mt * A_TILE + u * 32));
                            if (SPLIT) {
                                const uint64_t adl = desc_sw64(st + lo_off + (uint32_t)(mt * A_TILE + u * 32));
                                const uint64_t bdl = desc_plain(st + b_off + BLO + (uint32_t)(u * 2 * 128), 128, B_GROUP);
                                mma(acc + (uint32_t)(mt * NP), adl, bd, ID, (j | u) != 0);
                                mma(acc + (uint32_t)(mt * NP), ad, bdl, ID, 1);
                                mma(acc + (uint32_t)(mt * NP), ad, bd, ID, 1);
                            } else {
                                mma(acc + (uint32_t)(mt * NP), ad, bd, ID, (j | u) != 0);
                            }
                        }
                    }
                    commit(empty0 + 8 * s);
                }
                commit(accf0 + 8 * b);
            }
        }
    } else if (warp < 2 + GATHER_WARPS) {
        // ------------------------------------------------------- gather ---
        // gather warp g fills the B operand of every G-th stage: element
        // (c, k) at (c / 8) B_GROUP + (k / 4) 128 + (c % 8) 16 + (k % 4) 4 for
        // the stage's k = 0 .. KS - 1; lane (k % 4, c / 4 % 8).  G <= ST: a
        // warp waits on a stage's empty barrier only after its own previous
        // wait (G stages back) has seen the MMAs of ST - G <= 0 stages
        // earlier, so the barrier is never a full phase behind the parity
        // it polls for.
        constexpr int G = GATHER_WARPS < ST ? GATHER_WARPS : ST;
        const int g = warp - 2, kk = lane & 3, c4l = lane >> 2;
        constexpr int NE = (NP / 4 + 7) / 8;
        if (g >= G) goto done;
        int it = 0;
        for (int i = blockIdx.x; i < npatch; i += gridDim.x) {
            const int p = plist ? __ldg(plist + i) : i;
            const int s0 = poff[p], n = poff[p + 1] - s0, nst = (n + KS - 1) / KS;
            for (int j = 0; j < nst; ++j, ++it) {
                if (it % G != g) continue;
                const int s = it % ST;
                int dof[KS / 4];
#pragma unroll
                for (int k4 = 0; k4 < KS / 4; ++k4) {
                    const int k = j * KS + 4 * k4 + kk;
                    dof[k4] = k < n ? __ldg(pdofs + s0 + k) : -1;
                }
                float4 v[KS / 4][NE];
#pragma unroll
                for (int k4 = 0; k4 < KS / 4; ++k4)
#pragma unroll
                    for (int e = 0; e < NE; ++e) {
                        const int c = 4 * (c4l + 8 * e);
                        v[k4][e] = (dof[k4] >= 0 && c < M)
                                       ? __ldg(reinterpret_cast<const float4*>(X + (long long)dof[k4] * M + c))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                if (it >= ST && !mbar_wait(empty0 + 8 * s, ((it / ST) - 1) & 1, abort_flag)) goto done;
                unsigned char* bp = smem_tc + (stage0 - base) + (size_t)s * sbytes + b_off;
#pragma unroll
                for (int k4 = 0; k4 < KS / 4; ++k4) {
#pragma unroll
                    for (int e = 0; e < NE; ++e) {
                        const int c = 4 * (c4l + 8 * e);
                        if (c < NP) {
                            const float f[4] = {v[k4][e].x, v[k4][e].y, v[k4][e].z, v[k4][e].w};
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int cc = c + u;
                                const int o = (cc >> 3) * B_GROUP + k4 * 128 + (cc & 7) * 16 + kk * 4;
                                const uint32_t hi = to_tf32(f[u]);
                                *reinterpret_cast<uint32_t*>(bp + o) = hi;
                                if (SPLIT) *reinterpret_cast<uint32_t*>(bp + BLO + o) = to_tf32(f[u] - __uint_as_float(hi));
                            }
                        }
                    }
                }
                fence_proxy_async();
                mbar_arrive(full0 + 8 * s);
            }
        }
    } else {
        // ----------------------------------------------------- epilogue ---
        const int q = warp & 3;            // tensor-memory lanes 32 q .. 32 q + 31
        int pc = 0;
        for (int i = blockIdx.x; i < npatch; i += gridDim.x, ++pc) {
            const int p = plist ? __ldg(plist + i) : i;
            const int s0 = poff[p], n = poff[p + 1] - s0, tiles = tiles_of(n);
            const int b = pc % nbuf;
            float w[8];
#pragma unroll
            for (int mt = 0; mt < 8; ++mt) {
                const int row = mt * 128 + 32 * q + lane;
                w[mt] = (mt < tiles && row < n) ? __ldg(wt + __ldg(pdofs + s0 + row)) : 0.f;
            }
            if (!mbar_wait(accf0 + 8 * b, (pc / nbuf) & 1, abort_flag)) goto done;
            fence_after();
#pragma unroll
            for (int mt = 0; mt < 8; ++mt) {
                if (mt >= tiles) break;
                const int row = mt * 128 + 32 * q + lane;
#pragma unroll
                for (int cb = 0; cb < NP; cb += 16) {
                    uint32_t v[16];
                    ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * ccols + mt * NP + cb), v);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row < n && cb < M) {
                        float4* dst = reinterpret_cast<float4*>(Yb + (long long)(s0 + row) * M + cb);
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (cb + 4 * e < M)
                                dst[e] = make_float4(w[mt] * __uint_as_float(v[4 * e]), w[mt] * __uint_as_float(v[4 * e + 1]),
                                                     w[mt] * __uint_as_float(v[4 * e + 2]),
                                                     w[mt] * __uint_as_float(v[4 * e + 3]));
                    }
                }
            }
            fence_before();
            mbar_arrive(acce0 + 8 * b);
        }
    }
done:
    if (tid == 0 && *abort_flag) atomicExch(status, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace tc

__global__ void __launch_bounds__(256) k_pull_scatter(int n, int m, const int* __restrict__ soff,
                                                      const int* __restrict__ sidx, const float2* __restrict__ Yb,
                                                      float alpha, float beta, float2* __restrict__ out) {
    const int L = m >> 1;
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int j = (int)(gt / L), c2 = (int)(gt - (long long)j * L);
    if (j >= n) return;
    float2 acc = make_float2(0.f, 0.f);
    const int e = soff[j + 1];
    for (int q = soff[j]; q < e; ++q) {
        const float2 y = Yb[(long long)sidx[q] * L + c2];
        acc.x += y.x;
        acc.y += y.y;
    }
    const long long o = (long long)j * L + c2;
    if (beta == 0.f) out[o] = make_float2(alpha * acc.x, alpha * acc.y);
    else { const float2 v = out[o]; out[o] = make_float2(alpha * acc.x + beta * v.x, alpha * acc.y + beta * v.y); }
}

// thread per (row i, right-hand side c); a warp covers 32 right-hand sides
// of one row, so C's row is a broadcast and B's rows are coalesced
__global__ void __launch_bounds__(256) k_coarse_gemm(int nc, int ldc, int m, const double* __restrict__ C,
                                                     const float* __restrict__ B, float* __restrict__ E) {
    const long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int i = (int)(gt / m), c = (int)(gt - (long long)i * m);
    if (i >= nc) return;
    const double* ci = C + (long long)i * ldc;
    double s = 0.0;
    for (int j = 0; j < nc; ++j) s = fma(__ldg(ci + j), (double)__ldg(B + (long long)j * m + c), s);
    E[(long long)i * m + c] = (float)s;
}

}  // namespace

void to_interleaved(int n, int nrhs, int m, const double* r, float* X, cudaStream_t s) {
    k_to_interleaved<<<grid_of((long long)n * m, 256), 256, 0, s>>>(n, nrhs, m, r, X);
}

void from_interleaved(int n, int nrhs, int m, const float* X, double* z, cudaStream_t s) {
    k_from_interleaved<<<grid_of((long long)n * nrhs, 256), 256, 0, s>>>(n, nrhs, m, X, z);
}

void spmm(int mode, int nr, int m, const int* rp, const int* ci, const float* av, const float* X, float* Y,
          const float* B, cudaStream_t s) {
    const long long threads = (long long)nr * (m / 2);
    const int grid = (int)((threads + 255) / 256);
    const float2* X2 = reinterpret_cast<const float2*>(X);
    float2* Y2 = reinterpret_cast<float2*>(Y);
    const float2* B2 = reinterpret_cast<const float2*>(B);
    if (mode == 0) k_spmm<0><<<grid, 256, 0, s>>>(nr, m, rp, ci, av, X2, Y2, B2);
    else if (mode == 1) k_spmm<1><<<grid, 256, 0, s>>>(nr, m, rp, ci, av, X2, Y2, B2);
    else k_spmm<2><<<grid, 256, 0, s>>>(nr, m, rp, ci, av, X2, Y2, B2);
}

// warps per CTA: enough 16-row blocks per warp for the largest patch, at
// most 16 warps, spread evenly
int gemm_default_warps(int maxn) {
    const int nrb = (maxn + 15) / 16;
    const int per = (nrb + 15) / 16;
    return nrb <= 0 ? 1 : (nrb + per - 1) / per;
}

static size_t gemm_smem(int maxn, int m, int stages, int nw) {
    return sizeof(float) * ((size_t)m * rt_ld(maxn) + (size_t)nw * stages * SLOT);
}

template <int M, int MODE, int ST>
static void launch_gemm(int threads, size_t smem, int nlist, const int* plist, const int* poff, const int* pdofs,
                        const long long* ioff, const float* inv, const float* X, const float* wt, float* Yb,
                        cudaStream_t s) {
    cudaFuncSetAttribute(k_patch_gemm<M, MODE, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_patch_gemm<M, MODE, ST>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    k_patch_gemm<M, MODE, ST><<<nlist, threads, smem, s>>>(nlist, plist, poff, pdofs, ioff, inv, X, wt, Yb);
}

static int device_attr(cudaDeviceAttr attr) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, attr, dev);
    return v;
}

// nw warps per CTA (0: gemm_default_warps(maxn)); as many cp.async stages
// of 8, 6 or MIN_STAGES as fit the shared memory
template <int M, int MODE>
static void launch_gemm_st(int maxn, int nw, int nlist, const int* plist, const int* poff, const int* pdofs,
                           const long long* ioff, const float* inv, const float* X, const float* wt, float* Yb,
                           cudaStream_t s) {
    const size_t dev_max = (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin);
    if (nw <= 0) nw = gemm_default_warps(maxn);
    const int threads = 32 * nw;
    if (gemm_smem(maxn, M, 8, nw) <= dev_max)
        launch_gemm<M, MODE, 8>(threads, gemm_smem(maxn, M, 8, nw), nlist, plist, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else if (gemm_smem(maxn, M, 6, nw) <= dev_max)
        launch_gemm<M, MODE, 6>(threads, gemm_smem(maxn, M, 6, nw), nlist, plist, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else
        launch_gemm<M, MODE, MIN_STAGES>(threads, gemm_smem(maxn, M, MIN_STAGES, nw), nlist, plist, poff, pdofs, ioff,
                                         inv, X, wt, Yb, s);
}

// Patches of <= TC_MIN_N DoFs fill under half of a 128-row MMA tile; the
// warp-level kernel is faster there.  The 3xTF32 tensor-core kernel holds
// twice the operands per stage; up to TC_SPLIT_MAX_N DoFs (6 row tiles) two
// stages still fit.
constexpr int TC_MIN_N = 64, TC_SPLIT_MAX_N = 768;

int gemm_kind(int mode, int n) {
    if (n <= TC_MIN_N) return GEMM_KIND_WARP;
    if (mode == GEMM_TF32) return GEMM_KIND_TC;
    return n <= TC_SPLIT_MAX_N ? GEMM_KIND_TC : GEMM_KIND_WARP;
}

// tensor-core TF32 path: a persistent grid of one CTA per SM (the dynamic
// shared memory is at least half an SM's, so no two CTAs share an SM and its
// 512 tensor-memory columns), with as many pipeline stages as fit, at most 12
struct TcPlan { int stages = 0; size_t smem = 0; int grid = 0; };

static TcPlan tc_plan(int maxn, int m, int npatch, bool split = false) {
    TcPlan pl;
    const int np = tc::np_of(m);
    if (tc::tiles_of(maxn) > 8 || tc::tmem_cols(maxn, np) > 512) return pl;
    const long long optin = device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin);
    const long long per_sm = device_attr(cudaDevAttrMaxSharedMemoryPerMultiprocessor);
    const long long fixed = tc::HDR + 1024, sb = tc::stage_bytes(maxn, np, split);
    const long long st = std::min<long long>(12, (optin - fixed) / sb);
    if (st < 2) return pl;
    pl.stages = (int)st;
    pl.smem = (size_t)std::max<long long>(fixed + st * sb, per_sm / 2 + 1024);
    if ((long long)pl.smem > optin) pl.smem = (size_t)optin;
    pl.grid = std::max(1, std::min(npatch, device_attr(cudaDevAttrMultiProcessorCount)));
    return pl;
}

template <int M, int ST, bool SPLIT>
static void launch_tc(const TcPlan& pl, int nlist, const int* plist, int maxn, const int* poff, const int* pdofs,
                      const void* tmaps, const void* tmaps_lo, const float* X, const float* wt, float* Yb, int* status,
                      cudaStream_t s) {
    cudaFuncSetAttribute(tc::k_patch_gemm_tc<M, ST, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
    tc::k_patch_gemm_tc<M, ST, SPLIT><<<pl.grid, tc::THREADS, pl.smem, s>>>(
        nlist, maxn, plist, poff, pdofs, reinterpret_cast<const CUtensorMap*>(tmaps),
        reinterpret_cast<const CUtensorMap*>(tmaps_lo), X, wt, Yb, status);
}

template <int M, bool SPLIT>
static void launch_tc_st(int nlist, const int* plist, int maxn, const int* poff, const int* pdofs, const void* tmaps,
                         const void* tmaps_lo, const float* X, const float* wt, float* Yb, int* status, cudaStream_t s) {
    const TcPlan pl = tc_plan(maxn, M, nlist, SPLIT);
    switch (pl.stages) {
#define SBAT_TC_CASE(S) \
    case S: launch_tc<M, S, SPLIT>(pl, nlist, plist, maxn, poff, pdofs, tmaps, tmaps_lo, X, wt, Yb, status, s); break;
        SBAT_TC_CASE(2) SBAT_TC_CASE(3) SBAT_TC_CASE(4) SBAT_TC_CASE(5) SBAT_TC_CASE(6) SBAT_TC_CASE(7)
        SBAT_TC_CASE(8) SBAT_TC_CASE(9) SBAT_TC_CASE(10) SBAT_TC_CASE(11) SBAT_TC_CASE(12)
#undef SBAT_TC_CASE
        default: break;
    }
}

template <int M>
static void patch_gemm_m(int mode, int kind, int nw, int nlist, const int* plist, int maxn, const int* poff,
                         const int* pdofs, const long long* ioff, const float* inv, const void* tmaps,
                         const void* tmaps_hi, const void* tmaps_lo, const float* X, const float* wt, float* Yb,
                         int* status, cudaStream_t s) {
    if (kind == GEMM_KIND_AUTO) kind = gemm_kind(mode, maxn);
    if (kind == GEMM_KIND_TC && mode == GEMM_3XTF32)
        launch_tc_st<M, true>(nlist, plist, maxn, poff, pdofs, tmaps_hi, tmaps_lo, X, wt, Yb, status, s);
    else if (kind == GEMM_KIND_TC)
        launch_tc_st<M, false>(nlist, plist, maxn, poff, pdofs, tmaps, nullptr, X, wt, Yb, status, s);
    else if (mode == GEMM_3XTF32)
        launch_gemm_st<M, GEMM_3XTF32>(maxn, nw, nlist, plist, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else
        launch_gemm_st<M, GEMM_TF32>(maxn, nw, nlist, plist, poff, pdofs, ioff, inv, X, wt, Yb, s);
}

// the largest patch decides: a smaller patch of either kind needs no more
// shared or tensor memory than the largest one of that kind
const char* patch_gemm_check(int mode, int maxn, int m) {
    if (gemm_kind(mode, maxn) == GEMM_KIND_WARP)
        return gemm_smem(maxn, m, MIN_STAGES, gemm_default_warps(maxn)) <=
                       (size_t)device_attr(cudaDevAttrMaxSharedMemoryPerBlockOptin)
                   ? nullptr
                   : "patch too large for the shared memory of the warp-MMA patch GEMM at this width";
    if (tc::tiles_of(maxn) > 8 || tc::tmem_cols(maxn, tc::np_of(m)) > 512)
        return "patch too large for the tensor memory at this width";
    return tc_plan(maxn, m, 1, mode == GEMM_3XTF32).stages ? nullptr
                                                           : "patch too large for the shared memory of the tensor-core patch GEMM";
}

namespace {
__global__ void k_split_tf32(long long n, const float* __restrict__ a, float* __restrict__ hi, float* __restrict__ lo) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = a[i];
        const float h = __uint_as_float(to_tf32(x));
        hi[i] = h;
        lo[i] = x - h;
    }
}
}  // namespace

void split_tf32(long long n, const float* a, float* hi, float* lo, cudaStream_t s) {
    if (n > 0) k_split_tf32<<<grid_of(n, 256), 256, 0, s>>>(n, a, hi, lo);
}

int wait_probe(long long polls, int* result_dev, cudaStream_t s) {
    tc::k_wait_probe<<<1, 32, 0, s>>>(polls, result_dev);
    return (int)cudaGetLastError();
}

size_t tmap_bytes(int npatch) { return sizeof(CUtensorMap) * (size_t)std::max(npatch, 1); }

// One 2-D tensor map per patch over its FP32 inverse (inner extent ld =
// (n + 3) & ~3 floats, n rows of stride ld), box 16 x 128 with the 64-byte
// swizzle the MMA descriptors expect; zero fill outside.
void build_tmaps(int npatch, const int* poff_d, const long long* ioff_d, const float* inv_d, void* out_d) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            throw std::runtime_error("cuTensorMapEncodeTiled is not available");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    std::vector<int> poff(npatch + 1);
    std::vector<long long> ioff(npatch);
    if (cudaMemcpy(poff.data(), poff_d, sizeof(int) * (npatch + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(ioff.data(), ioff_d, sizeof(long long) * npatch, cudaMemcpyDeviceToHost) != cudaSuccess)
        throw std::runtime_error("patch offsets could not be read");
    std::vector<CUtensorMap> maps(npatch);
    for (int p = 0; p < npatch; ++p) {
        const int n = poff[p + 1] - poff[p], ld = (n + 3) & ~3;
        const cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)n};
        const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)tc::KS, 128u};
        const cuuint32_t estr[2] = {1u, 1u};
        const CUresult r = encode(&maps[p], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)(inv_d + ioff[p]), dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) throw std::runtime_error("cuTensorMapEncodeTiled failed for patch " + std::to_string(p));
    }
    if (cudaMemcpy(out_d, maps.data(), sizeof(CUtensorMap) * npatch, cudaMemcpyHostToDevice) != cudaSuccess)
        throw std::runtime_error("tensor maps could not be uploaded");
}

void patch_gemm(int mode, int kind, int nw, int nlist, const int* plist, int maxn, int m, const int* poff,
                const int* pdofs, const long long* ioff, const float* inv, const void* tmaps, const void* tmaps_hi,
                const void* tmaps_lo, const float* X, const float* wt, float* Yb, int* status, cudaStream_t s) {
    if (nlist <= 0) return;
    switch (m) {
#define SBAT_M(MM) \
    case MM: \
        patch_gemm_m<MM>(mode, kind, nw, nlist, plist, maxn, poff, pdofs, ioff, inv, tmaps, tmaps_hi, tmaps_lo, X, wt, \
                         Yb, status, s); \
        break;
        SBAT_M(8) SBAT_M(16) SBAT_M(32)
#undef SBAT_M
        default:
            patch_gemm_m<64>(mode, kind, nw, nlist, plist, maxn, poff, pdofs, ioff, inv, tmaps, tmaps_hi, tmaps_lo, X, wt,
                             Yb, status, s);
    }
}

void pull_scatter(int n, int m, const int* soff, const int* sidx, const float* Yb, float alpha, float beta,
                  float* out, cudaStream_t s) {
    const long long threads = (long long)n * (m / 2);
    k_pull_scatter<<<(int)((threads + 255) / 256), 256, 0, s>>>(n, m, soff, sidx, reinterpret_cast<const float2*>(Yb),
                                                                alpha, beta, reinterpret_cast<float2*>(out));
}

void coarse_gemm(int nc, int ldc, int m, const double* C, const float* B, float* E, cudaStream_t s) {
    const long long threads = (long long)nc * m;
    k_coarse_gemm<<<(int)((threads + 255) / 256), 256, 0, s>>>(nc, ldc, m, C, B, E);
}

}  // namespace sbat
