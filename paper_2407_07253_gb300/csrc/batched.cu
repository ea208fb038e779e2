// Kernels of the batched V-cycle; see batched.cuh.
#include "batched.cuh"

#include <cstdint>

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
__global__ void __launch_bounds__(512, 1) k_patch_gemm(int npatch, const int* __restrict__ poff,
                                                    const int* __restrict__ pdofs, const long long* __restrict__ ioff,
                                                    const float* __restrict__ inv, const float* __restrict__ X,
                                                    const float* __restrict__ wt, float* __restrict__ Yb) {
    extern __shared__ __align__(128) float smem_pg[];
    constexpr int NT = M / 8, Q = M / 4;
    const int p = blockIdx.x;
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
static int patch_gemm_warps(int maxn) {
    const int nrb = (maxn + 15) / 16;
    const int per = (nrb + 15) / 16;
    return nrb <= 0 ? 1 : (nrb + per - 1) / per;
}

static size_t gemm_smem(int maxn, int m, int stages) {
    return sizeof(float) * ((size_t)m * rt_ld(maxn) + (size_t)patch_gemm_warps(maxn) * stages * SLOT);
}

size_t patch_gemm_smem(int maxn, int m) { return gemm_smem(maxn, m, MIN_STAGES); }

template <int M, int MODE, int ST>
static void launch_gemm(int threads, size_t smem, int npatch, const int* poff, const int* pdofs,
                        const long long* ioff, const float* inv, const float* X, const float* wt, float* Yb,
                        cudaStream_t s) {
    cudaFuncSetAttribute(k_patch_gemm<M, MODE, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_patch_gemm<M, MODE, ST>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    k_patch_gemm<M, MODE, ST><<<npatch, threads, smem, s>>>(npatch, poff, pdofs, ioff, inv, X, wt, Yb);
}

template <int M, int MODE>
static void launch_gemm_st(int maxn, int npatch, const int* poff, const int* pdofs, const long long* ioff,
                           const float* inv, const float* X, const float* wt, float* Yb, cudaStream_t s) {
    static int dev_max = 0;
    if (dev_max == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    const int threads = 32 * patch_gemm_warps(maxn);
    if (gemm_smem(maxn, M, 8) <= (size_t)dev_max)
        launch_gemm<M, MODE, 8>(threads, gemm_smem(maxn, M, 8), npatch, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else if (gemm_smem(maxn, M, 6) <= (size_t)dev_max)
        launch_gemm<M, MODE, 6>(threads, gemm_smem(maxn, M, 6), npatch, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else
        launch_gemm<M, MODE, MIN_STAGES>(threads, gemm_smem(maxn, M, MIN_STAGES), npatch, poff, pdofs, ioff, inv, X,
                                         wt, Yb, s);
}

template <int M>
static void patch_gemm_m(int mode, int npatch, int maxn, const int* poff, const int* pdofs, const long long* ioff,
                         const float* inv, const float* X, const float* wt, float* Yb, cudaStream_t s) {
    if (mode == GEMM_3XTF32) launch_gemm_st<M, GEMM_3XTF32>(maxn, npatch, poff, pdofs, ioff, inv, X, wt, Yb, s);
    else launch_gemm_st<M, GEMM_TF32>(maxn, npatch, poff, pdofs, ioff, inv, X, wt, Yb, s);
}

void patch_gemm(int mode, int npatch, int maxn, int m, const int* poff, const int* pdofs, const long long* ioff,
                const float* inv, const float* X, const float* wt, float* Yb, cudaStream_t s) {
    switch (m) {
        case 8: patch_gemm_m<8>(mode, npatch, maxn, poff, pdofs, ioff, inv, X, wt, Yb, s); break;
        case 16: patch_gemm_m<16>(mode, npatch, maxn, poff, pdofs, ioff, inv, X, wt, Yb, s); break;
        case 32: patch_gemm_m<32>(mode, npatch, maxn, poff, pdofs, ioff, inv, X, wt, Yb, s); break;
        default: patch_gemm_m<64>(mode, npatch, maxn, poff, pdofs, ioff, inv, X, wt, Yb, s); break;
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
