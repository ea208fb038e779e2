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

// One CTA (4 warps) per patch.  The gathered block R_p (rows padded to a
// multiple of 8 with zeros, row stride m + 4 floats: conflict-free B
// fragments) sits in shared memory; warp w computes the 16-row blocks
// w, w + 4, ... of the product, streaming its rows of K_p^{-1} from HBM as
// A fragments (each inverse entry is read once, U k-steps in flight) and
// reusing every A fragment for the m / 8 column tiles.
//
// m16n8k8 TF32 fragments (g = lane / 4, t = lane % 4):
//   A (16 x 8, row): a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4)
//   B (8 x 8, col):  b0 (t, g), b1 (t + 4, g)
//   D (16 x 8):      d0 (g, 2t), d1 (g, 2t + 1), d2 (g + 8, 2t), d3 (g + 8, 2t + 1)
template <int M, int MODE>
__global__ void __launch_bounds__(128) k_patch_gemm(int npatch, const int* __restrict__ poff,
                                                    const int* __restrict__ pdofs, const long long* __restrict__ ioff,
                                                    const float* __restrict__ inv, const float* __restrict__ X,
                                                    const float* __restrict__ wt, float* __restrict__ Yb) {
    extern __shared__ float Rs[];
    constexpr int LD = M + 4, NT = M / 8, U = M >= 64 ? 4 : 8;
    const int p = blockIdx.x;
    const int s = poff[p], n = poff[p + 1] - s;
    const int n8 = (n + 7) & ~7, ld = (n + 3) & ~3;
    for (int idx = threadIdx.x; idx < n8 * M; idx += blockDim.x) {
        const int row = idx / M, c = idx - row * M;
        Rs[row * LD + c] = row < n ? X[(long long)pdofs[s + row] * M + c] : 0.0f;
    }
    __syncthreads();
    const float* A = inv + ioff[p];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int nrb = (n + 15) >> 4;
    for (int rb = warp; rb < nrb; rb += 4) {
        const int r0 = rb * 16 + g, r1 = r0 + 8;
        float d[NT][4];
#pragma unroll
        for (int q = 0; q < NT; ++q) d[q][0] = d[q][1] = d[q][2] = d[q][3] = 0.f;
        for (int kb = 0; kb < n8; kb += 8 * U) {
            float va[U][4];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int c0 = kb + 8 * u + t, c1 = c0 + 4;
                // A rows r0/r1, columns c0/c1 (zero outside the patch)
                va[u][0] = (r0 < n && c0 < n) ? __ldcs(A + (long long)c0 * ld + r0) : 0.f;
                va[u][1] = (r1 < n && c0 < n) ? __ldcs(A + (long long)c0 * ld + r1) : 0.f;
                va[u][2] = (r0 < n && c1 < n) ? __ldcs(A + (long long)c1 * ld + r0) : 0.f;
                va[u][3] = (r1 < n && c1 < n) ? __ldcs(A + (long long)c1 * ld + r1) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k0 = kb + 8 * u;
                if (k0 >= n8) break;
                uint32_t ah[4], al[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int x = 0; x < 4; ++x) ah[x] = to_tf32(va[u][x]);
                if (MODE == GEMM_3XTF32) {
#pragma unroll
                    for (int x = 0; x < 4; ++x) al[x] = to_tf32(va[u][x] - __uint_as_float(ah[x]));
                }
                const float* b0p = Rs + (k0 + t) * LD + g;
                const float* b1p = Rs + (k0 + t + 4) * LD + g;
#pragma unroll
                for (int q = 0; q < NT; ++q) {
                    const float x0 = b0p[q * 8], x1 = b1p[q * 8];
                    const uint32_t bh0 = to_tf32(x0), bh1 = to_tf32(x1);
                    if (MODE == GEMM_3XTF32) {
                        const uint32_t bl0 = to_tf32(x0 - __uint_as_float(bh0));
                        const uint32_t bl1 = to_tf32(x1 - __uint_as_float(bh1));
                        mma_tf32(d[q], al, bh0, bh1);
                        mma_tf32(d[q], ah, bl0, bl1);
                    }
                    mma_tf32(d[q], ah, bh0, bh1);
                }
            }
        }
        const float w0 = r0 < n ? wt[pdofs[s + r0]] : 0.f;
        const float w1 = r1 < n ? wt[pdofs[s + r1]] : 0.f;
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int c = q * 8 + 2 * t;
            if (r0 < n) *reinterpret_cast<float2*>(Yb + (long long)(s + r0) * M + c) = make_float2(w0 * d[q][0], w0 * d[q][1]);
            if (r1 < n) *reinterpret_cast<float2*>(Yb + (long long)(s + r1) * M + c) = make_float2(w1 * d[q][2], w1 * d[q][3]);
        }
    }
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

template <int M>
static void patch_gemm_m(int mode, int npatch, int maxn, const int* poff, const int* pdofs, const long long* ioff,
                         const float* inv, const float* X, const float* wt, float* Yb, cudaStream_t s) {
    const size_t smem = sizeof(float) * (size_t)((maxn + 7) & ~7) * (M + 4);
    if (mode == GEMM_3XTF32) {
        cudaFuncSetAttribute(k_patch_gemm<M, GEMM_3XTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_patch_gemm<M, GEMM_3XTF32><<<npatch, 128, smem, s>>>(npatch, poff, pdofs, ioff, inv, X, wt, Yb);
    } else {
        cudaFuncSetAttribute(k_patch_gemm<M, GEMM_TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_patch_gemm<M, GEMM_TF32><<<npatch, 128, smem, s>>>(npatch, poff, pdofs, ioff, inv, X, wt, Yb);
    }
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
