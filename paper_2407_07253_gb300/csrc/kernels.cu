// sm_103a kernels of the phMG hot path; declarations and roles in kernels.cuh.
#include "kernels.cuh"

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>

namespace skern {

__global__ void scale_by_inv(int n, const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y) {
    const double inv = 1.0 / s[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = x[i] * inv;
}

__global__ void sub_scalar(int n, double* __restrict__ x, const double* __restrict__ num, double den) {
    const double m = num[0] / den;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] -= m;
}

__global__ void sub_weighted(int n, double* __restrict__ x, const double* __restrict__ w, const double* __restrict__ num,
                             double den) {
    const double m = num[0] / den;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] -= w[i] * m;
}

__global__ void block_mass_inverse(int nc, int nb, const int* __restrict__ qcell, const double* __restrict__ minv,
                                   const double* __restrict__ scale, const double* __restrict__ y, double* __restrict__ z) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nc * nb;
         t += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(t / nb), a = (int)(t - (long long)e * nb);
        const int* q = qcell + (long long)e * nb;
        double acc = 0;
        for (int b = 0; b < nb; ++b) acc += minv[a * nb + b] * y[q[b]];
        z[q[a]] = scale[e] * acc;
    }
}

__global__ void csr_block_count(int nr, int nc, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ len) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        int c = 0;
        for (int p = rp[r]; p < rp[r + 1]; ++p) c += ci[p] < nc;
        len[r] = c;
    }
}

__global__ void csr_block_fill(int nr, int nc, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ v, const int* __restrict__ brp, int* __restrict__ bci,
                               double* __restrict__ bv, float* __restrict__ bv32) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nr; r += gridDim.x * blockDim.x) {
        int o = brp[r];
        for (int p = rp[r]; p < rp[r + 1]; ++p)
            if (ci[p] < nc) {
                bci[o] = ci[p];
                bv[o] = v[p];
                if (bv32) bv32[o] = (float)v[p];
                ++o;
            }
    }
}

// ------------------------------------------------------------ reductions ---
constexpr int MDOT_MAX = 32;

__global__ void __launch_bounds__(256) mdot_partial(int n, int m, const double* __restrict__ V, long long ldv,
                                                    const double* __restrict__ w, double* __restrict__ partial) {
    double acc[MDOT_MAX];
#pragma unroll
    for (int i = 0; i < MDOT_MAX; ++i) acc[i] = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double wk = w[k];
#pragma unroll
        for (int i = 0; i < MDOT_MAX; ++i)
            if (i < m) acc[i] += V[(long long)i * ldv + k] * wk;
    }
    __shared__ double red[8][MDOT_MAX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < MDOT_MAX; ++i) {
        if (i >= m) break;
        double v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < m) {
        double s = 0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += red[wv][threadIdx.x];
        partial[(long long)blockIdx.x * m + threadIdx.x] = s;
    }
}

__global__ void mdot_final(int nblocks, int m, const double* __restrict__ partial, double* __restrict__ out,
                           double* __restrict__ acc, int sqrt_out) {
    const int i = threadIdx.x;
    if (i >= m) return;
    double s = 0;
    for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * m + i];
    if (acc) acc[i] += s;
    out[i] = (sqrt_out && i == 0) ? sqrt(s) : s;
}

// Fused multi-dots: every block writes its partial sums, the last block to
// finish (atomic ticket) adds them in a fixed order, so results are bitwise
// reproducible.  Launched with MDOT_BLOCKS blocks of MDOT_THREADS threads.

// Block partial sums of a[0..m) (and, if with_extra, of `extra` as column
// m) into partial[blockIdx.x][0..m + with_extra).  The threads' values go to
// shared memory 16 columns at a time and one warp sums a column (8 adds per
// lane, then 5 shuffle steps): FP64 adds are scarce on this GPU, and this
// takes ~13 warp instructions per column instead of 5 per warp and column
// for a shuffle tree in every warp.
template <int MM>
__device__ __forceinline__ void mdot_block_partials(int m, const double (&a)[MM], double extra, bool with_extra,
                                                    double* partial) {
    constexpr int NT = MDOT_THREADS, CH = 16;
    __shared__ double red[CH][NT];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = NT >> 5;
    const int mc = m + (with_extra ? 1 : 0);
#pragma unroll
    for (int c0 = 0; c0 < MM + 1; c0 += CH) {
        if (c0 >= mc) break;
#pragma unroll
        for (int q = 0; q < CH; ++q) {
            const int c = c0 + q;
            if (c < MM && c < m) red[q][t] = a[c < MM ? c : 0];
            else if (with_extra && c == m) red[q][t] = extra;
        }
        __syncthreads();
        for (int q = warp; q < CH && c0 + q < mc; q += nw) {
            double sum = 0.0;
#pragma unroll
            for (int j = 0; j < NT / 32; ++j) sum += red[q][lane + 32 * j];
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
            if (lane == 0) partial[(long long)blockIdx.x * mc + c0 + q] = sum;
        }
        __syncthreads();
    }
}

// true in the last block to arrive (which then resets the ticket)
__device__ __forceinline__ bool mdot_last_block(unsigned int* ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// last block: out[i] = sum_b partial[b][i] (i < mcols <= 32, row stride
// mcols) over the grid's blocks in a fixed order (MDOT_THREADS / 32 threads
// per output, strided, then a fixed shuffle tree), with acc[i] += out[i] for
// i < macc; the partials are read from L2 (ld.global.cg), all loads issued
// together
__device__ __forceinline__ void mdot_reduce_partials(int mcols, int macc, const double* partial, double* out,
                                                     double* acc, int sqrt_out, unsigned int* ticket) {
    constexpr int G = MDOT_THREADS / 32;
    const int i = threadIdx.x / G, sub = threadIdx.x % G;
    double s = 0;
    if (i < mcols) {
        double t[(MDOT_BLOCKS + G - 1) / G];
#pragma unroll
        for (int q = 0; q < (MDOT_BLOCKS + G - 1) / G; ++q) {
            const int b = sub + G * q;
            t[q] = b < (int)gridDim.x ? __ldcg(partial + (long long)b * mcols + i) : 0.0;
        }
#pragma unroll
        for (int q = 0; q < (MDOT_BLOCKS + G - 1) / G; ++q) s += t[q];
    }
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (i < mcols && sub == 0) {
        if (acc && i < macc) acc[i] += s;
        out[i] = (sqrt_out && i == 0) ? sqrt(s) : s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// The accumulators are unrolled to MM (>= m): FP64 FMAs are scarce on this
// GPU, so the host picks the smallest MM in {4, 8, 16, 32} that holds m.
template <int MM>
__global__ void __launch_bounds__(MDOT_THREADS) mdot_fused_t(int n, int m, const double* __restrict__ V, long long ldv,
                                                    const double* __restrict__ w, double* __restrict__ partial,
                                                    unsigned int* __restrict__ ticket, double* __restrict__ out,
                                                    double* __restrict__ acc, int sqrt_out) {
    double a[MM];
#pragma unroll
    for (int i = 0; i < MM; ++i) a[i] = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const double wk = w[k];
#pragma unroll
        for (int i = 0; i < MM; ++i)
            if (i < m) a[i] = fma(V[(long long)i * ldv + k], wk, a[i]);
    }
    mdot_block_partials(m, a, 0.0, false, partial);
    if (!mdot_last_block(ticket)) return;
    mdot_reduce_partials(m, acc ? m : 0, partial, out, acc, sqrt_out, ticket);
}

void mdot_fused(int n, int m, const double* V, long long ldv, const double* w, double* partial, unsigned int* ticket,
                double* out, double* acc, int sqrt_out, cudaStream_t s) {
    if (m <= 4) mdot_fused_t<4><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, w, partial, ticket, out, acc, sqrt_out);
    else if (m <= 8) mdot_fused_t<8><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, w, partial, ticket, out, acc, sqrt_out);
    else if (m <= 16) mdot_fused_t<16><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, w, partial, ticket, out, acc, sqrt_out);
    else mdot_fused_t<32><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, w, partial, ticket, out, acc, sqrt_out);
}

// Second classical Gram-Schmidt pass fused with the first pass's update:
//   w <- w - V h  (h = the first pass's coefficients),
//   out[0..m) = V^T w,  out[m] = w^T w  (of the updated w),  acc[i] += out[i].
// m <= MDOT_MAX - 1.
template <int MM>
__global__ void __launch_bounds__(MDOT_THREADS) maxpy_mdot_t(int n, int m, const double* __restrict__ V, long long ldv,
                                                    const double* __restrict__ h, double* __restrict__ w,
                                                    double* __restrict__ partial, unsigned int* __restrict__ ticket,
                                                    double* __restrict__ out, double* __restrict__ acc) {
    __shared__ double hs[MDOT_MAX];
    if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    double a[MM], nrm = 0.0;
#pragma unroll
    for (int i = 0; i < MM; ++i) a[i] = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double wk = w[k];
        if constexpr (MM <= 16) {
            // few vectors: keep V[.][k] in registers between the two uses
            double vk[MM];
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < m) { vk[i] = V[(long long)i * ldv + k]; wk = fma(-hs[i], vk[i], wk); }
            w[k] = wk;
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < m) a[i] = fma(vk[i], wk, a[i]);
        } else {
            // many vectors: the second read hits L1
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < m) wk = fma(-hs[i], V[(long long)i * ldv + k], wk);
            w[k] = wk;
#pragma unroll
            for (int i = 0; i < MM; ++i)
                if (i < m) a[i] = fma(V[(long long)i * ldv + k], wk, a[i]);
        }
        nrm = fma(wk, wk, nrm);
    }
    mdot_block_partials(m, a, nrm, true, partial);
    if (!mdot_last_block(ticket)) return;
    mdot_reduce_partials(m + 1, m, partial, out, acc, 0, ticket);
}

void maxpy_mdot(int n, int m, const double* V, long long ldv, const double* h, double* w, double* partial,
                unsigned int* ticket, double* out, double* acc, cudaStream_t s) {
    if (m <= 4) maxpy_mdot_t<4><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, h, w, partial, ticket, out, acc);
    else if (m <= 8) maxpy_mdot_t<8><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, h, w, partial, ticket, out, acc);
    else if (m <= 16) maxpy_mdot_t<16><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, h, w, partial, ticket, out, acc);
    else maxpy_mdot_t<31><<<MDOT_BLOCKS, MDOT_THREADS, 0, s>>>(n, m, V, ldv, h, w, partial, ticket, out, acc);
}

// Last update of classical Gram-Schmidt, normalised:
//   w <- (w - V h) / nu,  nu = sqrt(max(nrm2 - sum_i h_i^2, 0)),  *hn = nu,
// where nrm2 = ||w||^2 before the update (Pythagoras: the second pass's h is
// O(eps) relative to w, so the difference loses no accuracy).
__global__ void __launch_bounds__(256) maxpy_normalise(int n, int m, const double* __restrict__ V, long long ldv,
                                                       const double* __restrict__ h, const double* __restrict__ nrm2,
                                                       double* __restrict__ w, double* __restrict__ hn) {
    __shared__ double hs[MDOT_MAX];
    __shared__ double sinv;
    if (threadIdx.x < m) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        double q = *nrm2;
        for (int i = 0; i < m; ++i) q -= hs[i] * hs[i];
        const double nu = sqrt(q > 0.0 ? q : 0.0);
        sinv = 1.0 / nu;
        if (blockIdx.x == 0) *hn = nu;
    }
    __syncthreads();
    const double inv = sinv;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double s = w[k];
        for (int i = 0; i < m; ++i) s -= hs[i] * V[(long long)i * ldv + k];
        w[k] = s * inv;
    }
}

__global__ void __launch_bounds__(256) maxpy(int n, int m, const double* __restrict__ V, long long ldv,
                                             const double* __restrict__ h, double sign, double* __restrict__ w) {
    __shared__ double hs[MDOT_MAX];
    if (threadIdx.x < m) hs[threadIdx.x] = sign * h[threadIdx.x];
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        double s = w[k];
        for (int i = 0; i < m; ++i) s += hs[i] * V[(long long)i * ldv + k];
        w[k] = s;
    }
}

// ------------------------------------------------------ DoF -> slot map ---
// For the patch index list pdofs[0..nent): the slots q of every DoF j in
// increasing order (soff / sidx, the pull scatter's summation order) and the
// partition-of-unity weight 1 / (number of patches holding j).
__global__ void slot_count(long long nent, const int* __restrict__ pdofs, int* __restrict__ cnt) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nent; q += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[pdofs[q]], 1);
}
__global__ void slot_fill(long long nent, const int* __restrict__ pdofs, const int* __restrict__ soff, int* __restrict__ cur,
                          int* __restrict__ sidx) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nent; q += (long long)gridDim.x * blockDim.x) {
        const int j = pdofs[q];
        sidx[soff[j] + atomicAdd(&cur[j], 1)] = (int)q;
    }
}
__global__ void slot_sort(int n, const int* __restrict__ soff, int* __restrict__ sidx, double* __restrict__ wt) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int* a = sidx + soff[j];
        const int len = soff[j + 1] - soff[j];
        for (int x = 1; x < len; ++x) {
            const int v = a[x];
            int y = x;
            for (; y > 0 && a[y - 1] > v; --y) a[y] = a[y - 1];
            a[y] = v;
        }
        wt[j] = len ? 1.0 / len : 0.0;
    }
}

// -------------------------------------------------------------- patches ---
__global__ void __launch_bounds__(256) patch_gather(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                                    const long long* __restrict__ moff, const int* __restrict__ rp,
                                                    const int* __restrict__ ci, const double* __restrict__ av,
                                                    double* __restrict__ out) {
    extern __shared__ int sdofs[];
    const int p = blockIdx.x;
    const int s = poff[p], n = poff[p + 1] - s;
    for (int a = threadIdx.x; a < n; a += blockDim.x) sdofs[a] = pdofs[s + a];
    __syncthreads();
    double* M = out + moff[p];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int a = warp; a < n; a += nw) {
        const int g = sdofs[a];
        const int e = rp[g + 1];
        for (int q = rp[g] + lane; q < e; q += 32) {
            const int c = ci[q];
            int lo = 0, hi = n - 1;
            while (lo < hi) {              // first position with sdofs[pos] >= c
                const int mid = (lo + hi) >> 1;
                if (sdofs[mid] < c) lo = mid + 1; else hi = mid;
            }
            if (sdofs[lo] == c) M[(long long)a * n + lo] = av[q];
        }
    }
}

// In-place Gauss-Jordan with partial pivoting on a row-major n x n matrix A
// (shared or global memory).  The first maximum |A[i][k]|, i >= k, is the
// pivot; rows are swapped, the pivot row scaled, column k eliminated from all
// other rows; at the end columns are swapped back in reverse order.  Returns
// (in *status) 0, or 1 + the step of the first zero pivot.
__device__ void gj_core(double* A, int n, double* colk, int* ipiv, int* status) {
    __shared__ double s_val[32];
    __shared__ int s_idx[32];
    __shared__ int s_p;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    int bad = 0;
    for (int k = 0; k < n; ++k) {
        // pivot search: each warp scans a strided subset, then warp 0 reduces
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += nt) {
            const double v = fabs(A[(long long)i * n + k]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            const int nw = nt >> 5;
            best = lane < nw ? s_val[lane] : -1.0;
            bi = lane < nw ? s_idx[lane] : n;
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) {
                if (!(best > 0.0) || bi >= n) { bi = k; if (!bad) bad = k + 1; }
                s_p = bi;
                ipiv[k] = bi;
                if (bad && *status == 0) *status = bad;
            }
        }
        __syncthreads();
        const int p = s_p;
        if (p != k)
            for (int j = tid; j < n; j += nt) {
                const double t = A[(long long)k * n + j];
                A[(long long)k * n + j] = A[(long long)p * n + j];
                A[(long long)p * n + j] = t;
            }
        __syncthreads();
        const double piv = A[(long long)k * n + k];
        const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
        for (int i = tid; i < n; i += nt) colk[i] = A[(long long)i * n + k];
        __syncthreads();
        for (int j = tid; j < n; j += nt) A[(long long)k * n + j] = (j == k) ? inv : A[(long long)k * n + j] * inv;
        __syncthreads();
        // rank-1 elimination of column k from every other row
        int i = tid / n, j = tid - (tid / n) * n;
        const int step_i = nt / n, step_j = nt - step_i * n;
        for (; i < n;) {
            if (i != k) {
                const double f = colk[i];
                if (j == k) A[(long long)i * n + k] = -f * inv;
                else A[(long long)i * n + j] -= f * A[(long long)k * n + j];
            }
            i += step_i;
            j += step_j;
            if (j >= n) { j -= n; ++i; }
        }
        __syncthreads();
    }
    // undo the row interchanges by column interchanges in reverse order
    for (int k = n - 1; k >= 0; --k) {
        const int p = ipiv[k];
        if (p != k)
            for (int i = tid; i < n; i += nt) {
                const double t = A[(long long)i * n + k];
                A[(long long)i * n + k] = A[(long long)i * n + p];
                A[(long long)i * n + p] = t;
            }
        __syncthreads();
    }
}

__device__ void gj_store(const double* A, int n, double* inv64, long long o64, float* inv32, long long o32) {
    const int ld64 = (n + 1) & ~1, ld32 = (n + 3) & ~3;
    if (inv64)
        for (int t = threadIdx.x; t < ld64 * n; t += blockDim.x) {
            const int j = t / ld64, i = t - j * ld64;
            inv64[o64 + t] = i < n ? A[(long long)i * n + j] : 0.0;
        }
    if (inv32)
        for (int t = threadIdx.x; t < ld32 * n; t += blockDim.x) {
            const int j = t / ld32, i = t - j * ld32;
            inv32[o32 + t] = i < n ? (float)A[(long long)i * n + j] : 0.0f;
        }
}

__global__ void __launch_bounds__(256) gj_inverse_smem(int npatch, const int* __restrict__ poff, const long long* __restrict__ moff,
                                                       double* __restrict__ work, const long long* __restrict__ off64,
                                                       double* __restrict__ inv64, const long long* __restrict__ off32,
                                                       float* __restrict__ inv32, int* __restrict__ status, int) {
    extern __shared__ double smem[];
    const int p = blockIdx.x;
    const int n = poff[p + 1] - poff[p];
    if (n > GJ_SMEM_MAX_N || n == 0) return;
    double* A = smem;
    double* colk = smem + (long long)n * n;
    int* ipiv = (int*)(colk + n);
    __shared__ int st;
    if (threadIdx.x == 0) st = 0;
    const double* W = work + moff[p];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = W[t];
    __syncthreads();
    gj_core(A, n, colk, ipiv, &st);
    __syncthreads();
    gj_store(A, n, inv64, off64 ? off64[p] : 0, inv32, off32 ? off32[p] : 0);
    // keep the row-major inverse in the workspace for export
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) work[moff[p] + t] = A[t];
    if (threadIdx.x == 0) status[p] = st;
}

__global__ void __launch_bounds__(512) gj_inverse_global(int npatch, const int* __restrict__ poff, const long long* __restrict__ moff,
                                                         double* __restrict__ work, const long long* __restrict__ off64,
                                                         double* __restrict__ inv64, const long long* __restrict__ off32,
                                                         float* __restrict__ inv32, int* __restrict__ status,
                                                         int* __restrict__ ipiv_ws, double* __restrict__ col_ws) {
    const int p = blockIdx.x;
    const int n = poff[p + 1] - poff[p];
    if (n <= GJ_SMEM_MAX_N) return;
    __shared__ int st;
    if (threadIdx.x == 0) st = 0;
    __syncthreads();
    double* A = work + moff[p];
    gj_core(A, n, col_ws + poff[p], ipiv_ws + poff[p], &st);
    __syncthreads();
    gj_store(A, n, inv64, off64 ? off64[p] : 0, inv32, off32 ? off32[p] : 0);
    if (threadIdx.x == 0) status[p] = st;
}

// Sign flip of a double through its bit pattern: no floating-point
// instruction (the FP64 pipe is the bottleneck of the patch inversion).
__device__ __forceinline__ double flip(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}

// Row-pair mapping of an upper triangle: warp w takes rows w and n-1-w, whose
// (n - w) + (w + 1) = n + 1 entries fill its lanes evenly; entry l of the pair
// is (i, j).  Returns the entry count of the pair.
__device__ __forceinline__ int pair_len(int n, int pr) { return (pr == n - 1 - pr) ? n - pr : n + 1; }
__device__ __forceinline__ void pair_entry(int n, int pr, int l, int& i, int& j) {
    const int len0 = n - pr;
    if (l < len0) { i = pr; j = pr + l; }
    else { i = n - 1 - pr; j = i + (l - len0); }
}

// Goodnight's symmetric sweep of an SPD matrix in full row-major storage
// (leading dimension lda), updating the upper triangle.  Sweeping pivot k maps
//   a_kk -> -1/a_kk,  a_ik -> a_ik/a_kk (i != k),  a_ij -> a_ij - a_ik a_kj / a_kk,
// and sweeping every pivot in order leaves -A^{-1}.  An SPD matrix needs no
// pivoting.  On return the full matrix holds +A^{-1} (upper triangle negated
// and mirrored by sign-bit flips).  Every updated entry costs exactly one FMA:
// the pivot column is published scaled (cs) and unscaled (ck), and the lane
// that updates the next diagonal entry forms the next reciprocal, so a pivot
// needs two barriers.  Scratch: ck[2n] (double-buffered column), cs[n],
// rinv[2].  status <- 1 + step of the first non-positive pivot.
__device__ void sweep_spd(double* A, int n, int lda, double* ck, double* cs, double* rinv, int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int npair = (n + 1) >> 1;
    if (tid == 0) {
        const double piv = A[0];
        if (!(piv > 0.0) && *status == 0) *status = 1;
        rinv[0] = piv > 0.0 ? 1.0 / piv : 0.0;
    }
    for (int i = tid; i < n; i += nt) ck[i] = A[i];
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        const double* ckc = ck + (k & 1) * n;
        double* ckn = ck + ((k + 1) & 1) * n;
        const double inv = rinv[k & 1];
        for (int i = tid; i < n; i += nt) cs[i] = ckc[i] * inv;
        __syncthreads();
        for (int pr = warp; pr < npair; pr += nw) {
            const int tot = pair_len(n, pr);
            for (int l = lane; l < tot; l += 32) {
                int i, j;
                pair_entry(n, pr, l, i, j);
                double* a = A + (long long)i * lda + j;
                double v = fma(-cs[i], ckc[j], *a);
                if (i == k || j == k) v = (i == j) ? flip(inv) : cs[i == k ? j : i];
                *a = v;
                // publish column k+1 of the updated matrix for the next pivot
                if (j == k + 1) ckn[i] = v;
                else if (i == k + 1) ckn[j] = v;
                if (i == k + 1 && j == k + 1) {
                    if (!(v > 0.0) && *status == 0) *status = k + 2;
                    rinv[(k + 1) & 1] = v > 0.0 ? 1.0 / v : 0.0;
                }
            }
        }
        __syncthreads();
    }
    // -A^{-1} (upper) -> +A^{-1} (full)
    for (int pr = warp; pr < npair; pr += nw) {
        const int tot = pair_len(n, pr);
        for (int l = lane; l < tot; l += 32) {
            int i, j;
            pair_entry(n, pr, l, i, j);
            const double v = flip(A[(long long)i * lda + j]);
            A[(long long)i * lda + j] = v;
            A[(long long)j * lda + i] = v;
        }
    }
    __syncthreads();
}

// sweep_spd two pivots per step: the same two FMAs per entry and pivot pair,
// in the same order, with the same special cases, so the result is bit for
// bit that of sweep_spd, with half the block barriers.  Warp 0 prepares a
// step from the published columns k and k+1 (both before pivot k): the
// scaled column cs = col_k / a_kk, column k+1 after pivot k (each entry by
// the operation its owner would apply, so c1p equals the column sweep_spd
// would publish), its scaled copy cs1 and the two reciprocals; then every
// entry is swept by pivot k and pivot k+1, and the owners of columns k+2 and
// k+3 publish them for the next step.  Scratch: ck[4n] (two column pairs,
// double-buffered), cs[n], c1p[n], cs1[n], rinv[2].  status <- 1 + step of
// the first non-positive pivot.  PP: A is the pair-packed upper triangle
// (pp_row; lda unused), which the sweep touches in its own order, and on
// return holds +A^{-1} there (negated in place, not mirrored).
template <bool PP>
__device__ void sweep_spd2(double* A, int n, int lda, double* ck, double* cs, double* c1p, double* cs1, double* rinv,
                           int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int npair = (n + 1) >> 1;
    for (int i = tid; i < n; i += nt) {
        // column 0 = row 0, column 1 = (0, 1) then row 1
        if (PP) {
            ck[i] = A[i];
            if (n > 1) ck[n + i] = i == 0 ? A[1] : A[pp_row(n, 1) + i];
        } else {
            ck[i] = A[i];
            if (n > 1) ck[n + i] = i == 0 ? A[1] : A[(long long)lda + i];
        }
    }
    __syncthreads();
    for (int k = 0, b = 0; k < n; k += 2, ++b) {
        const double* col0 = ck + (b & 1) * 2 * n;                 // column k before pivot k
        const double* col1 = col0 + n;                             // column k+1 before pivot k
        double* nx0 = ck + ((b + 1) & 1) * 2 * n;                  // columns k+2, k+3 for the next step
        double* nx1 = nx0 + n;
        const bool two = k + 1 < n;
        if (warp == 0) {
            const double akk = col0[k];
            double inv0 = 0.0;
            if (lane == 0) {
                if (!(akk > 0.0) && *status == 0) *status = k + 1;
                inv0 = akk > 0.0 ? 1.0 / akk : 0.0;
            }
            inv0 = __shfl_sync(0xffffffffu, inv0, 0);
            double csk1 = 0.0, p1 = 0.0, inv1 = 0.0;
            if (two) {
                csk1 = col0[k + 1] * inv0;
                p1 = fma(-csk1, col0[k + 1], col1[k + 1]);         // (k+1, k+1) after pivot k
                if (lane == 0) {
                    if (!(p1 > 0.0) && *status == 0) *status = k + 2;
                    inv1 = p1 > 0.0 ? 1.0 / p1 : 0.0;
                }
                inv1 = __shfl_sync(0xffffffffu, inv1, 0);
            }
            for (int i = lane; i < n; i += 32) {
                const double csi = col0[i] * inv0;
                cs[i] = csi;
                if (two) {
                    double v;
                    if (i == k) v = csk1;                                         // (k, k+1)
                    else if (i < k + 1) v = fma(-csi, col0[k + 1], col1[i]);      // (i, k+1)
                    else if (i == k + 1) v = p1;                                  // (k+1, k+1)
                    else v = fma(-csk1, col0[i], col1[i]);                        // (k+1, i)
                    c1p[i] = v;
                    cs1[i] = v * inv1;
                }
            }
            if (lane == 0) {
                rinv[0] = inv0;
                rinv[1] = inv1;
            }
        }
        __syncthreads();
        const double inv0 = rinv[0], inv1 = rinv[1];
        for (int pr = warp; pr < npair; pr += nw) {
            const int tot = pair_len(n, pr);
            for (int l = lane; l < tot; l += 32) {
                int i, j;
                pair_entry(n, pr, l, i, j);
                double* a = PP ? A + (long long)pr * (n + 1) + l : A + (long long)i * lda + j;
                double v = fma(-cs[i], col0[j], *a);
                if (i == k || j == k) v = (i == j) ? flip(inv0) : cs[i == k ? j : i];
                if (two) {
                    const int k1 = k + 1;
                    double w = fma(-cs1[i], c1p[j], v);
                    if (i == k1 || j == k1) w = (i == j) ? flip(inv1) : cs1[i == k1 ? j : i];
                    v = w;
                }
                *a = v;
                if (j == k + 2) nx0[i] = v;
                else if (i == k + 2) nx0[j] = v;
                if (j == k + 3) nx1[i] = v;
                else if (i == k + 3) nx1[j] = v;
            }
        }
        __syncthreads();
    }
    // -A^{-1} (upper) -> +A^{-1} (full, or the packed upper triangle)
    for (int pr = warp; pr < npair; pr += nw) {
        const int tot = pair_len(n, pr);
        for (int l = lane; l < tot; l += 32) {
            if (PP) {
                double* a = A + (long long)pr * (n + 1) + l;
                *a = flip(*a);
            } else {
                int i, j;
                pair_entry(n, pr, l, i, j);
                const double v = flip(A[(long long)i * lda + j]);
                A[(long long)i * lda + j] = v;
                A[(long long)j * lda + i] = v;
            }
        }
    }
    __syncthreads();
}

// Block inverse of one Vanka patch with the saddle structure
//   K_i = [L 0 .. B_0^T; 0 L .. B_1^T; ..; B_0 B_1 .. 0]
// (the d velocity components share the SPD block L on the same nodes):
//   Li = L^{-1}, W_c = Li B_c^T, S = sum_c B_c W_c, Si = S^{-1}, X_c = W_c Si,
//   K_i^{-1} = [blockdiag(Li) - X W^T, X; X^T, -Si].
// Li and Si come from the symmetric sweep.  Products map one output entry
// to one thread (a warp's lanes share few rows), the symmetric velocity block
// uses the row-pair mapping, so FP64 instructions run with full warps.  The
// (symmetric) inverse is formed on its upper triangle and every value written
// to both of its positions: column-major padded FP64 / FP32 and, if back,
// row-major into K.
// Factored form (fac64 / fac32, VEC = 2 / 4): per patch, column-major with
// leading dimensions rounded up to VEC, padding zero:
//   Li [ldl][nv]  (ldl = nv up to VEC), W [ldw][np] (ldw = d nv up to VEC),
//   Si [lds][np]  (lds = np up to VEC),
// from which K_i^{-1} r = (blockdiag(Li) r_u + W s, -s), s = Si (r_p - W^T r_u)
// (saddle_apply).  With no explicit output (inv64, inv32 NULL, back 0) the
// products X = W Si and blockdiag(Li) - X W^T are skipped.
__device__ void saddle_core(int d, int n, int nv, double* K, double* scratch, double* inv64, float* inv32,
                            double* fac64, float* fac32, int back, int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int np = n - d * nv, npp = np | 1, dnv = d * nv;
    const int mx = nv > np ? nv : np;
    double* Ls = scratch;                          // [nv][nv]
    double* Bt = Ls + (long long)nv * nv;          // [c][a][q], becomes X
    double* Wm = Bt + (long long)d * nv * npp;     // [c][a][q]
    double* Ss = Wm + (long long)d * nv * npp;     // [q][r]
    double* ck = Ss + (long long)np * np;          // [2][mx]
    double* cs = ck + 2 * mx;                      // [mx]
    double* rinv = cs + mx;                        // [2]
    for (int i = warp; i < nv; i += nw)
        for (int j = i + lane; j < nv; j += 32) Ls[i * nv + j] = K[(long long)i * n + j];
    for (int r = warp; r < dnv; r += nw)
        for (int q = lane; q < np; q += 32) Bt[(long long)r * npp + q] = K[(long long)r * n + dnv + q];
    __syncthreads();
    sweep_spd(Ls, nv, nv, ck, cs, rinv, status);
    const bool fac = fac64 || fac32;
    const int ldl = fac64 ? (nv + 1) & ~1 : (nv + 3) & ~3;
    const int ldw = fac64 ? (dnv + 1) & ~1 : (dnv + 3) & ~3;
    const int lds = fac64 ? (np + 1) & ~1 : (np + 3) & ~3;
    if (fac) {
        // Li (symmetric, full after the sweep)
        const int tot = nv * ldl;
        for (int t = tid; t < tot; t += nt) {
            const int b = t / ldl, a = t - b * ldl;
            const double v = a < nv ? Ls[a * nv + b] : 0.0;
            if (fac64) fac64[t] = v;
            if (fac32) fac32[t] = (float)v;
        }
    }
    // W_c = Li B_c^T: entry t = (r, q), r = c nv + a
    const int nw_out = dnv * np;
    for (int t = tid; t < nw_out; t += nt) {
        const int r = t / np, q = t - r * np;
        const int c = r / nv, a = r - c * nv;
        const double* li = Ls + a * nv;
        const double* bt = Bt + (long long)c * nv * npp + q;
        double s = 0.0;
        for (int b = 0; b < nv; ++b) s = fma(li[b], bt[(long long)b * npp], s);
        Wm[(long long)r * npp + q] = s;
    }
    __syncthreads();
    if (fac) {
        const long long o = (long long)ldl * nv;
        const int tot = np * ldw;
        for (int t = tid; t < tot; t += nt) {
            const int q = t / ldw, r = t - q * ldw;
            const double v = r < dnv ? Wm[(long long)r * npp + q] : 0.0;
            if (fac64) fac64[o + t] = v;
            if (fac32) fac32[o + t] = (float)v;
        }
    }
    // S = sum_c B_c W_c, upper triangle q <= r
    const int ns = np * (np + 1) / 2;
    for (int t = tid; t < ns; t += nt) {
        int q = 0, rem = t;
        while (rem >= np - q) { rem -= np - q; ++q; }
        const int r = q + rem;
        double s = 0.0;
        for (int a = 0; a < dnv; ++a) s = fma(Bt[(long long)a * npp + q], Wm[(long long)a * npp + r], s);
        Ss[q * np + r] = s;
    }
    __syncthreads();
    sweep_spd(Ss, np, np, ck, cs, rinv, status);
    if (fac) {
        const long long o = (long long)ldl * nv + (long long)ldw * np;
        const int tot = np * lds;
        for (int t = tid; t < tot; t += nt) {
            const int r = t / lds, q = t - r * lds;
            const double v = q < np ? Ss[q * np + r] : 0.0;
            if (fac64) fac64[o + t] = v;
            if (fac32) fac32[o + t] = (float)v;
        }
    }
    if (!inv64 && !inv32 && !back) return;      // factored form only
    // X_c = W_c Si (overwrites Bt)
    for (int t = tid; t < nw_out; t += nt) {
        const int r = t / np, q = t - r * np;
        const double* w = Wm + (long long)r * npp;
        double s = 0.0;
        for (int x = 0; x < np; ++x) s = fma(w[x], Ss[x * np + q], s);
        Bt[(long long)r * npp + q] = s;
    }
    __syncthreads();
    const int ld64 = (n + 1) & ~1, ld32 = (n + 3) & ~3;
    auto put = [&](int i, int j, double v) {
        if (inv64) { inv64[(long long)j * ld64 + i] = v; inv64[(long long)i * ld64 + j] = v; }
        if (inv32) { inv32[(long long)j * ld32 + i] = (float)v; inv32[(long long)i * ld32 + j] = (float)v; }
        if (back) { K[(long long)i * n + j] = v; K[(long long)j * n + i] = v; }
    };
    // velocity block: blockdiag(Li) - X W^T, upper triangle by row pairs
    const int vpairs = (dnv + 1) >> 1;
    for (int pr = warp; pr < vpairs; pr += nw) {
        const int tot = pair_len(dnv, pr);
        for (int l = lane; l < tot; l += 32) {
            int i, j;
            pair_entry(dnv, pr, l, i, j);
            const int c = i / nv, a = i - c * nv, c2 = j / nv, b = j - c2 * nv;
            const double* x = Bt + (long long)i * npp;
            const double* w = Wm + (long long)j * npp;
            double v = c == c2 ? Ls[a * nv + b] : 0.0;
            for (int q = 0; q < np; ++q) v = fma(-x[q], w[q], v);
            put(i, j, v);
        }
    }
    // velocity-pressure block X and pressure block -Si (copies)
    for (int t = tid; t < nw_out; t += nt) {
        const int r = t / np, q = t - r * np;
        put(r, dnv + q, Bt[(long long)r * npp + q]);
    }
    for (int t = tid; t < ns; t += nt) {
        int q = 0, rem = t;
        while (rem >= np - q) { rem -= np - q; ++q; }
        put(dnv + q, dnv + q + rem, flip(Ss[q * np + q + rem]));
    }
    // zero the padding rows of the column-major copies
    for (int j = tid; j < n; j += nt) {
        if (inv64)
            for (int i = n; i < ld64; ++i) inv64[(long long)j * ld64 + i] = 0.0;
        if (inv32)
            for (int i = n; i < ld32; ++i) inv32[(long long)j * ld32 + i] = 0.0f;
    }
}

// The factored form alone (no explicit output), in less shared memory: the
// components' B_c^T and W_c = Li B_c^T go through one pair of buffers, W_c
// is written out as soon as it exists and S = sum_c B_c W_c accumulates over
// the components.  Scratch: saddle_scratch_factored(d, n, nv, PP) doubles.
// position of global DoF c in a patch's sorted DoF list sd[0 .. n), or -1
__device__ __forceinline__ int patch_pos(const int* sd, int n, int c) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sd[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    return sd[lo] == c ? lo : -1;
}

// K == nullptr: the blocks are read from the CSR operator (rp, ci, av) rows
// of the patch's DoFs sd (sorted, shared memory) instead of a dense copy:
// the velocity block of component 0 (its upper triangle) and, per component,
// B_c^T, each entry placed by a binary search of its column in sd
template <bool PP>
__device__ void saddle_core_factored(int d, int n, int nv, const double* K, const int* sd, const int* __restrict__ rp,
                                     const int* __restrict__ ci, const double* __restrict__ av, double* scratch,
                                     double* fac64, float* fac32, int packed, int* status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const int np = n - d * nv, npp = np | 1, dnv = d * nv;
    const int mx = nv > np ? nv : np;
    double* Ls = scratch;                          // PP: pair-packed upper triangle (pp_row), else [nv][nv]
    double* Bt = Ls + (PP ? pp_size(nv) : (long long)nv * nv);   // [a][q] of the current component
    double* Wm = Bt + (long long)nv * npp;         // [a][q] of the current component
    double* Ss = Wm + (long long)nv * npp;         // [q][r]
    double* ck = Ss + (long long)np * np;          // [4][mx] (sweep_spd2's column pairs)
    double* cs = ck + 4 * mx;                      // [mx]
    double* c1p = cs + mx;                         // [mx]
    double* cs1 = c1p + mx;                        // [mx]
    double* rinv = cs1 + mx;                       // [2]
    // [np][mw]: bit a of column q set where B_c^T[a][q] != 0; the products
    // with B_c^T visit those rows only, in increasing order (the skipped
    // terms are exact zeros, so the sums equal the dense ones), which saves
    // most of the DFMAs of W and S: B couples a pressure node only with the
    // velocity nodes of the cells in its support
    const int mw = (nv + 63) >> 6;
    unsigned long long* mk = reinterpret_cast<unsigned long long*>(rinv + 2);
    const int vec = fac64 ? 2 : 4;
    const int ldl = (nv + vec - 1) / vec * vec;
    const int ldw = (dnv + vec - 1) / vec * vec;
    const int lds = (np + vec - 1) / vec * vec;
    const long long lenL = packed ? ((long long)nv * (nv + 1) / 2 + vec - 1) / vec * vec : (long long)ldl * nv;
    const long long oW = lenL, oS = oW + (long long)ldw * np;
    const int ns = np * (np + 1) / 2;
    if (K) {
        for (int i = warp; i < nv; i += nw)
            for (int j = i + lane; j < nv; j += 32) Ls[(PP ? pp_row(nv, i) : i * nv) + j] = K[(long long)i * n + j];
    } else {
        // the rows of component 0 give the velocity block and B_0^T
        for (int t = tid; t < (PP ? pp_size(nv) : (long long)nv * nv); t += nt) Ls[t] = 0.0;
        for (int t = tid; t < nv * npp; t += nt) Bt[t] = 0.0;
        __syncthreads();
        for (int i = warp; i < nv; i += nw) {
            const int g = sd[i], e = rp[g + 1];
            for (int q = rp[g] + lane; q < e; q += 32) {
                const int pos = patch_pos(sd, n, ci[q]);
                if (pos >= i && pos < nv) Ls[(PP ? pp_row(nv, i) : i * nv) + pos] = av[q];
                else if (pos >= dnv) Bt[(long long)i * npp + pos - dnv] = av[q];
            }
        }
    }
    for (int t = tid; t < np * np; t += nt) Ss[t] = 0.0;
    __syncthreads();
    sweep_spd2<PP>(Ls, nv, nv, ck, cs, c1p, cs1, rinv, status);
    if (packed) {
        // upper triangle row by row: (a, b >= a) at a nv - a (a - 1) / 2 + b - a
        for (int a = warp; a < nv; a += nw) {
            const long long o = (long long)a * nv - (long long)a * (a - 1) / 2 - a;
            const int ra = PP ? pp_row(nv, a) : a * nv;
            for (int b = a + lane; b < nv; b += 32) {
                const double v = Ls[ra + b];
                if (fac64) fac64[o + b] = v;
                if (fac32) fac32[o + b] = (float)v;
            }
        }
        for (long long t = (long long)nv * (nv + 1) / 2 + tid; t < lenL; t += nt) {
            if (fac64) fac64[t] = 0.0;
            if (fac32) fac32[t] = 0.0f;
        }
    } else {
        const int tot = nv * ldl;
        for (int t = tid; t < tot; t += nt) {
            const int b = t / ldl, a = t - b * ldl;
            const double v = a >= nv ? 0.0 : PP ? Ls[a <= b ? pp_row(nv, a) + b : pp_row(nv, b) + a] : Ls[a * nv + b];
            if (fac64) fac64[t] = v;
            if (fac32) fac32[t] = (float)v;
        }
    }
    {
        // W's padding rows
        for (int t = tid; t < np * (ldw - dnv); t += nt) {
            const int q = t / (ldw - dnv), r = dnv + t - q * (ldw - dnv);
            if (fac64) fac64[oW + (long long)q * ldw + r] = 0.0;
            if (fac32) fac32[oW + (long long)q * ldw + r] = 0.0f;
        }
    }
    for (int c = 0; c < d; ++c) {
        if (K) {
            for (int a = warp; a < nv; a += nw)
                for (int q = lane; q < np; q += 32) Bt[(long long)a * npp + q] = K[(long long)(c * nv + a) * n + dnv + q];
        } else if (c > 0) {
            for (int t = tid; t < nv * npp; t += nt) Bt[t] = 0.0;
            __syncthreads();
            for (int a = warp; a < nv; a += nw) {
                const int g = sd[c * nv + a], e = rp[g + 1];
                for (int q = rp[g] + lane; q < e; q += 32) {
                    const int pos = patch_pos(sd, n, ci[q]);
                    if (pos >= dnv) Bt[(long long)a * npp + pos - dnv] = av[q];
                }
            }
        }
        __syncthreads();
        // nonzero rows of every column of B_c^T (a warp per column)
        for (int q = warp; q < np; q += nw)
            for (int w = 0; w < mw; ++w) {
                const int a0 = w * 64 + lane, a1 = a0 + 32;
                const unsigned lo = __ballot_sync(0xffffffffu, a0 < nv && Bt[(long long)a0 * npp + q] != 0.0);
                const unsigned hi = __ballot_sync(0xffffffffu, a1 < nv && Bt[(long long)a1 * npp + q] != 0.0);
                if (lane == 0) mk[q * mw + w] = ((unsigned long long)hi << 32) | lo;
            }
        __syncthreads();
        // W_c = Li B_c^T: a warp takes column q for 32 rows a, so that its
        // lanes share q's mask (one trip count: FP64 instructions are issued
        // for the whole warp); Li is symmetric, read along row b
        const int nh = (nv + 31) >> 5;
        for (int it = warp; it < np * nh; it += nw) {
            const int q = it / nh, a = (it - q * nh) * 32 + lane;
            const int ra = PP ? pp_row(nv, a) : 0;
            const double* bt = Bt + q;
            double sacc = 0.0;
            for (int w = 0; w < mw; ++w)
                for (unsigned long long m = mk[q * mw + w]; m; m &= m - 1) {
                    const int b = w * 64 + __ffsll((long long)m) - 1;
                    if (a < nv)
                        sacc = fma(Ls[PP ? (b <= a ? pp_row(nv, b) + a : ra + b) : b * nv + a], bt[(long long)b * npp], sacc);
                }
            if (a < nv) Wm[(long long)a * npp + q] = sacc;
        }
        __syncthreads();
        for (int t = tid; t < nv * np; t += nt) {
            const int q = t / nv, a = t - q * nv;
            const double v = Wm[(long long)a * npp + q];
            if (fac64) fac64[oW + (long long)q * ldw + c * nv + a] = v;
            if (fac32) fac32[oW + (long long)q * ldw + c * nv + a] = (float)v;
        }
        // S += B_c W_c on the upper triangle q <= r (each entry one thread)
        for (int t = tid; t < ns; t += nt) {
            int q = 0, rem = t;
            while (rem >= np - q) { rem -= np - q; ++q; }
            const int r = q + rem;
            double sacc = 0.0;
            for (int w = 0; w < mw; ++w)
                for (unsigned long long m = mk[q * mw + w]; m; m &= m - 1) {
                    const int a = w * 64 + __ffsll((long long)m) - 1;
                    sacc = fma(Bt[(long long)a * npp + q], Wm[(long long)a * npp + r], sacc);
                }
            Ss[q * np + r] += sacc;
        }
        __syncthreads();
    }
    sweep_spd2<false>(Ss, np, np, ck, cs, c1p, cs1, rinv, status);
    {
        const int tot = np * lds;
        for (int t = tid; t < tot; t += nt) {
            const int r = t / lds, q = t - r * lds;
            const double v = q < np ? Ss[q * np + r] : 0.0;
            if (fac64) fac64[oS + t] = v;
            if (fac32) fac32[oS + t] = (float)v;
        }
    }
}

__global__ void __launch_bounds__(256) saddle_inverse_smem(int npatch, int d, const int* __restrict__ poff,
                                                           const int* __restrict__ pnv, const long long* __restrict__ moff,
                                                           double* __restrict__ work, const long long* __restrict__ off64,
                                                           double* __restrict__ inv64, const long long* __restrict__ off32,
                                                           float* __restrict__ inv32, const long long* __restrict__ foff64,
                                                           double* __restrict__ fac64, const long long* __restrict__ foff32,
                                                           float* __restrict__ fac32, int back, int packed,
                                                           long long max_scratch, const int* __restrict__ pdofs,
                                                           const int* __restrict__ rp, const int* __restrict__ ci,
                                                           const double* __restrict__ av, int sd_off,
                                                           int* __restrict__ status) {
    extern __shared__ double sscr[];
    const int p = blockIdx.x;
    const int n = poff[p + 1] - poff[p], nv = pnv[p];
    if (n == 0 || saddle_scratch(d, n, nv) > max_scratch) return;
    __shared__ int st;
    int* sd = reinterpret_cast<int*>(sscr + sd_off);
    if (!work && (inv64 || inv32 || back)) {      // the explicit forms need the dense block
        if (threadIdx.x == 0) status[p] = 1;
        return;
    }
    if (threadIdx.x == 0) st = 0;
    if (!work)
        for (int a = threadIdx.x; a < n; a += blockDim.x) sd[a] = pdofs[poff[p] + a];
    __syncthreads();
    if (!inv64 && !inv32 && !back)
        saddle_core_factored<true>(d, n, nv, work ? work + moff[p] : nullptr, sd, rp, ci, av, sscr,
                             fac64 ? fac64 + foff64[p] : nullptr, fac32 ? fac32 + foff32[p] : nullptr, packed, &st);
    else
        saddle_core(d, n, nv, work + moff[p], sscr, inv64 ? inv64 + off64[p] : nullptr,
                    inv32 ? inv32 + off32[p] : nullptr, fac64 ? fac64 + foff64[p] : nullptr,
                    fac32 ? fac32 + foff32[p] : nullptr, back, &st);
    __syncthreads();
    if (threadIdx.x == 0) status[p] = st;
}

__global__ void __launch_bounds__(256) saddle_inverse_global(int npatch, int d, const int* __restrict__ poff,
                                                             const int* __restrict__ pnv, const long long* __restrict__ moff,
                                                             double* __restrict__ work, const long long* __restrict__ off64,
                                                             double* __restrict__ inv64, const long long* __restrict__ off32,
                                                             float* __restrict__ inv32, const long long* __restrict__ foff64,
                                                             double* __restrict__ fac64, const long long* __restrict__ foff32,
                                                             float* __restrict__ fac32, int back, int packed,
                                                             long long max_scratch, const long long* __restrict__ soff,
                                                             double* __restrict__ scratch, int* __restrict__ status) {
    const int p = blockIdx.x;
    const int n = poff[p + 1] - poff[p], nv = pnv[p];
    if (n == 0 || saddle_scratch(d, n, nv) <= max_scratch) return;
    __shared__ int st;
    if (threadIdx.x == 0) st = 0;
    __syncthreads();
    if (!inv64 && !inv32 && !back)
        saddle_core_factored<false>(d, n, nv, work + moff[p], nullptr, nullptr, nullptr, nullptr, scratch + soff[p],
                             fac64 ? fac64 + foff64[p] : nullptr, fac32 ? fac32 + foff32[p] : nullptr, packed, &st);
    else
        saddle_core(d, n, nv, work + moff[p], scratch + soff[p], inv64 ? inv64 + off64[p] : nullptr,
                    inv32 ? inv32 + off32[p] : nullptr, fac64 ? fac64 + foff64[p] : nullptr,
                    fac32 ? fac32 + foff32[p] : nullptr, back, &st);
    __syncthreads();
    if (threadIdx.x == 0) status[p] = st;
}

// One ASM sweep.  The patch inverse is column-major with its leading
// dimension padded to VEC rows; a thread owns VEC consecutive rows (one
// 16-byte vector per column) and the columns are split among G groups of
// row-owners (G = blockDim / row groups), each thread keeping 8 independent
// 16-byte loads in flight.  The groups' partial sums are added in shared
// memory in a fixed order.  The gathered residual of the patch sits in
// shared memory.
template <typename T, typename V, int VEC>
__device__ __forceinline__ void patch_apply_body(int p, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                                 const long long* __restrict__ ioff, const T* __restrict__ inv,
                                                 const T* __restrict__ r, const T* __restrict__ wt, T* __restrict__ Y,
                                                 T* xs, V* red) {
    const int s = poff[p], n = poff[p + 1] - s;
    const int ldv = (n + VEC - 1) / VEC;
    for (int a = threadIdx.x; a < n; a += blockDim.x) xs[a] = r[pdofs[s + a]];
    __syncthreads();
    const int G = ldv >= (int)blockDim.x ? 1 : (int)blockDim.x / ldv;
    const V* base = reinterpret_cast<const V*>(inv + ioff[p]);
    for (int t0 = 0; t0 < ldv; t0 += blockDim.x) {          // more row groups than threads: loop
        const int t = threadIdx.x;
        const int rg = t0 + (G == 1 ? t : t % ldv), g = G == 1 ? 0 : t / ldv;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (g < G && rg < ldv) {
            const V* col = base + rg;
            int j = g;
            for (; j + 7 * G < n; j += 8 * G) {
                V v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcs(col + (long long)(j + u * G) * ldv);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const T x = xs[j + u * G];
                    if constexpr (VEC == 4) { a0 += v[u].x * x; a1 += v[u].y * x; a2 += v[u].z * x; a3 += v[u].w * x; }
                    else { a0 += v[u].x * x; a1 += v[u].y * x; }
                }
            }
            for (; j < n; j += G) {
                const V v = __ldcs(col + (long long)j * ldv);
                const T x = xs[j];
                if constexpr (VEC == 4) { a0 += v.x * x; a1 += v.y * x; a2 += v.z * x; a3 += v.w * x; }
                else { a0 += v.x * x; a1 += v.y * x; }
            }
        }
        if (G > 1) {
            if (g < G && rg < ldv) {
                V o;
                if constexpr (VEC == 4) o = V{a0, a1, a2, a3};
                else o = V{a0, a1};
                red[g * ldv + (rg - t0)] = o;
            }
            __syncthreads();
            if (t < ldv) {
                V o = red[t];
                for (int gg = 1; gg < G; ++gg) {
                    const V q = red[gg * ldv + t];
                    if constexpr (VEC == 4) { o.x += q.x; o.y += q.y; o.z += q.z; o.w += q.w; }
                    else { o.x += q.x; o.y += q.y; }
                }
                if constexpr (VEC == 4) { a0 = o.x; a1 = o.y; a2 = o.z; a3 = o.w; }
                else { a0 = o.x; a1 = o.y; }
            }
        }
        if (g == 0 && rg < ldv) {
            const int row0 = VEC * rg;
            const T out[4] = {a0, a1, a2, a3};
#pragma unroll
            for (int q = 0; q < VEC; ++q)
                if (row0 + q < n) Y[s + row0 + q] = wt[pdofs[s + row0 + q]] * out[q];
        }
        if (G > 1) __syncthreads();
    }
}

__global__ void __launch_bounds__(128) patch_apply_f32(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                                       const long long* __restrict__ ioff, const float* __restrict__ inv,
                                                       const float* __restrict__ r, const float* __restrict__ wt,
                                                       float* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smem_pa[];
    float4* red = reinterpret_cast<float4*>(smem_pa);
    float* xs = reinterpret_cast<float*>(smem_pa + sizeof(float4) * (blockDim.x + 4));
    pdl_wait();
    pdl_release();
    patch_apply_body<float, float4, 4>(blockIdx.x, poff, pdofs, ioff, inv, r, wt, Y, xs, red);
}

__global__ void __launch_bounds__(128) patch_apply_f64(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                                       const long long* __restrict__ ioff, const double* __restrict__ inv,
                                                       const double* __restrict__ r, const double* __restrict__ wt,
                                                       double* __restrict__ Y) {
    extern __shared__ __align__(16) unsigned char smem_pa[];
    double2* red = reinterpret_cast<double2*>(smem_pa);
    double* xs = reinterpret_cast<double*>(smem_pa + sizeof(double2) * (blockDim.x + 4));
    pdl_wait();
    pdl_release();
    patch_apply_body<double, double2, 2>(blockIdx.x, poff, pdofs, ioff, inv, r, wt, Y, xs, red);
}

// One ASM sweep with factored saddle inverses (saddle_core's factored form):
//   t = r_p - W^T r_u,  s = Si t,  z_u = blockdiag(Li) r_u + W s,  z_p = -s,
//   Y[poff[i] + a] = w[dof_a] z_a.
// One CTA of SADDLE_APPLY_THREADS threads per patch.  The gathered residual
// and W are staged in shared memory (W is used twice); Li is streamed from
// HBM once, as in patch_apply_body: a thread owns VEC consecutive rows and
// accumulates them for the d components at once, G groups of row owners
// split the columns, eight 16-byte loads in flight per thread, the groups'
// partial sums added in a fixed order.
__device__ __forceinline__ float vcomp(const float4& v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }
__device__ __forceinline__ double vcomp(const double2& v, int e) { return e == 0 ? v.x : v.y; }
__device__ __forceinline__ float4 mkvec(const float* a, float4*) { return make_float4(a[0], a[1], a[2], a[3]); }
__device__ __forceinline__ double2 mkvec(const double* a, double2*) { return make_double2(a[0], a[1]); }

template <typename T, typename V, int VEC>
__device__ __forceinline__ void saddle_apply_body(int p, int d, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                                  const int* __restrict__ pnv, const long long* __restrict__ foff,
                                                  const T* __restrict__ fac, const T* __restrict__ r,
                                                  const T* __restrict__ wt, T* __restrict__ Y, int xs_len, int ws_len,
                                                  unsigned char* smem) {
    constexpr int NT = SADDLE_APPLY_THREADS;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int s0 = poff[p], n = poff[p + 1] - s0, nv = pnv[p], dnv = d * nv, np = n - dnv;
    if (n == 0) return;
    const int ldl = (nv + VEC - 1) / VEC * VEC, ldw = (dnv + VEC - 1) / VEC * VEC;
    const T* Li = fac + foff[p];
    const T* Wg = Li + (long long)ldl * nv;
    const T* Sg = Wg + (long long)ldw * np;
    V* red = reinterpret_cast<V*>(smem);                         // [NT][3]
    T* ws = reinterpret_cast<T*>(smem + sizeof(V) * NT * 3);     // [ws_len]   W, column-major
    T* xs = ws + ws_len;                                         // [xs_len]   gathered r
    T* ys = xs + xs_len;                                         // [xs_len]   blockdiag(Li) r_u
    T* tq = ys + xs_len;                                         // [xs_len]   t
    T* sq = tq + xs_len;                                         // [xs_len]   s
    for (int a = tid; a < n; a += NT) xs[a] = r[pdofs[s0 + a]];
    // W is staged in shared memory when the level's largest fits (ws_len > 0),
    // else both of its uses read it from global memory (the second from cache)
    const T* wsrc = ws_len > 0 ? ws : Wg;
    if (ws_len > 0) {
        const V* wv = reinterpret_cast<const V*>(Wg);
        V* wsv = reinterpret_cast<V*>(ws);
        const int nvec = ldw * np / VEC;
        for (int t = tid; t < nvec; t += NT) wsv[t] = __ldcs(wv + t);
    }
    __syncthreads();
    // t = r_p - W^T r_u: one warp per pressure row, lanes over the velocity DoFs
    for (int q = warp; q < np; q += NT / 32) {
        const T* wc = wsrc + (long long)q * ldw;
        T acc = 0;
        for (int a = lane; a < dnv; a += 32) acc += wc[a] * xs[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) tq[q] = xs[dnv + q] - acc;
    }
    __syncthreads();
    // s = Si t (Si symmetric: entry (q, x) at Sg[x * lds + q]) and
    // y_c = Li r_c for every component c
    const int lds = (np + VEC - 1) / VEC * VEC;
    for (int q = tid; q < np; q += NT) {
        T acc = 0;
        for (int x = 0; x < np; ++x) acc += __ldcs(Sg + (long long)x * lds + q) * tq[x];
        sq[q] = acc;
    }
    const int ldv = ldl / VEC;
    const int G = ldv >= NT ? 1 : NT / ldv;
    const V* base = reinterpret_cast<const V*>(Li);
    for (int t0 = 0; t0 < ldv; t0 += NT) {
        const int rg = t0 + (G == 1 ? tid : tid % ldv), g = G == 1 ? 0 : tid / ldv;
        T acc[3][VEC];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[c][u] = 0;
        const bool own = g < G && rg < ldv;
        if (own) {
            const V* col = base + rg;
            int b = g;
            for (; b + 7 * G < nv; b += 8 * G) {
                V v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = __ldcs(col + (long long)(b + u * G) * ldv);
#pragma unroll
                for (int u = 0; u < 8; ++u)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        if (c < d) {
                            const T x = xs[c * nv + b + u * G];
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[c][e] += vcomp(v[u], e) * x;
                        }
                    }
            }
            for (; b < nv; b += G) {
                const V v = __ldcs(col + (long long)b * ldv);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (c < d) {
                        const T x = xs[c * nv + b];
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[c][e] += vcomp(v, e) * x;
                    }
            }
        }
        if (G > 1) {
            if (own)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (c < d) red[(g * ldv + (rg - t0)) * 3 + c] = mkvec(acc[c], (V*)nullptr);
            __syncthreads();
            if (tid < ldv) {
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (c < d) {
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[c][e] = vcomp(red[tid * 3 + c], e);
                        for (int gg = 1; gg < G; ++gg) {
                            const V q = red[(gg * ldv + tid) * 3 + c];
#pragma unroll
                            for (int e = 0; e < VEC; ++e) acc[c][e] += vcomp(q, e);
                        }
                    }
            }
        }
        if (g == 0 && rg < ldv) {
            const int row0 = VEC * rg;
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (c < d)
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (row0 + e < nv) ys[c * nv + row0 + e] = acc[c][e];
        }
        __syncthreads();
    }
    // z_u = y + W s, z_p = -s, weighted
    for (int a = tid; a < dnv; a += NT) {
        T z = ys[a];
        for (int q = 0; q < np; ++q) z += wsrc[(long long)q * ldw + a] * sq[q];
        Y[s0 + a] = wt[pdofs[s0 + a]] * z;
    }
    for (int q = tid; q < np; q += NT) Y[s0 + dnv + q] = -wt[pdofs[s0 + dnv + q]] * sq[q];
}

__global__ void __launch_bounds__(SADDLE_APPLY_THREADS) saddle_apply_f32(
    int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pdofs, const int* __restrict__ pnv,
    const long long* __restrict__ foff, const float* __restrict__ fac, const float* __restrict__ r,
    const float* __restrict__ wt, float* __restrict__ Y, int xs_len, int ws_len) {
    extern __shared__ __align__(16) unsigned char smem_sa[];
    pdl_wait();
    pdl_release();
    saddle_apply_body<float, float4, 4>(blockIdx.x, d, poff, pdofs, pnv, foff, fac, r, wt, Y, xs_len, ws_len, smem_sa);
}

__global__ void __launch_bounds__(SADDLE_APPLY_THREADS) saddle_apply_f64(
    int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pdofs, const int* __restrict__ pnv,
    const long long* __restrict__ foff, const double* __restrict__ fac, const double* __restrict__ r,
    const double* __restrict__ wt, double* __restrict__ Y, int xs_len, int ws_len) {
    extern __shared__ __align__(16) unsigned char smem_sa[];
    pdl_wait();
    pdl_release();
    saddle_apply_body<double, double2, 2>(blockIdx.x, d, poff, pdofs, pnv, foff, fac, r, wt, Y, xs_len, ws_len, smem_sa);
}

// ---- the same sweep with each patch's factored block brought into shared
// memory by one bulk copy (cp.async.bulk, completion on an mbarrier) -------
// One CTA of SA_BULK_THREADS threads per patch: thread 0 issues the copy of
// the patch's (packed Li, W, Si) block (contiguous, a multiple of 16 bytes)
// while the others gather the residual and the partition-of-unity weights
// of the patch's DoFs; every product then reads shared memory (reading W and
// Si from global memory instead, to fit more CTAs per SM, measured slower:
// 42 us against 38 us per level-0 sweep of the bench problem):
//   t = r_p - W^T r_u   (one warp per pressure row, lanes over the velocity rows)
//   y_c = Li r_c        (one thread per velocity row and component)
//   s = Si t            (one thread per pressure row)
//   z_u = y + W s, z_p = -s, weighted.
// The wait on the copy is bounded: after SA_WAIT_LIMIT polls the
// CTA sets *status = 1, waits (bounded) for the copy once more and returns.
__device__ __forceinline__ uint32_t sa_smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void sa_mbar_init(uint32_t a) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool sa_mbar_try(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void sa_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void saddle_apply_bulk_body(
    int d, const int* __restrict__ poff, const int* __restrict__ pdofs, const int* __restrict__ pnv,
    const long long* __restrict__ foff, const T* __restrict__ fac, const T* __restrict__ r,
    const T* __restrict__ wt, T* __restrict__ Y, int buf_bytes, int xs_len, int* __restrict__ status,
    unsigned char* smem, unsigned long long* bar) {
    constexpr int NT = SA_BULK_THREADS;
    constexpr int VEC = 16 / sizeof(T);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = blockIdx.x;
    T* xs = reinterpret_cast<T*>(smem + (size_t)buf_bytes);   // [xs_len] gathered r
    T* wq = xs + xs_len;                                       // [xs_len] weights
    T* ys = wq + xs_len;                                       // [xs_len] y
    T* tq = ys + xs_len;                                       // [xs_len] t
    T* sq = tq + xs_len;                                       // [xs_len] s
    const uint32_t b = sa_smem_u32(bar);
    const int s0 = poff[p], n = poff[p + 1] - s0, nv = pnv[p], dnv = d * nv, np = n - dnv;
    const int lenL = (nv * (nv + 1) / 2 + VEC - 1) / VEC * VEC;
    // the factors are constant: their copy starts before the wait for the
    // kernel that wrote r (programmatic dependent launch)
    if (tid == 0) {
        sa_mbar_init(b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const long long o = foff[p];
        const uint32_t bytes = (uint32_t)((foff[p + 1] - o) * (long long)sizeof(T));
        if (bytes > 0) sa_bulk_load(sa_smem_u32(smem), fac + o, bytes, b);
        else asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
    }
    pdl_wait();
    pdl_release();
    for (int a = tid; a < n; a += NT) {
        const int j = pdofs[s0 + a];
        xs[a] = r[j];
        wq[a] = wt[j];
    }
    // the barrier's initialisation (thread 0) is ordered before anyone polls
    // it by this __syncthreads; then warp 0 alone polls it (bounded: polling
    // by every warp took issue slots from the other CTAs on the SM), the
    // others wait at the block barrier and test the completed phase once
    __syncthreads();
    bool ok = warp != 0;
    if (warp == 0)
        for (long long it = 0; it < SA_WAIT_LIMIT; ++it)
            if (sa_mbar_try(b, 0)) { ok = true; break; }
    if (__syncthreads_and(ok) && warp != 0) ok = sa_mbar_try(b, 0);
    if (!__syncthreads_and(ok)) {
        if (tid == 0) {
            for (long long it = 0; it < SA_WAIT_LIMIT && !sa_mbar_try(b, 0); ++it) {}
            atomicExch(status, 1);
        }
        return;
    }
    const int ldw = (dnv + VEC - 1) / VEC * VEC;
    const int lds = (np + VEC - 1) / VEC * VEC;
    const T* Lp = reinterpret_cast<const T*>(smem);            // Li, packed upper triangle
    const T* Wm = Lp + lenL;
    const T* Si = Wm + ldw * np;
    for (int q = warp; q < np; q += NT / 32) {
        const T* wc = Wm + q * ldw;
        T acc = 0;
        for (int a = lane; a < dnv; a += 32) acc += wc[a] * xs[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) tq[q] = xs[dnv + q] - acc;
    }
    // y_c = Li r_c: Li[a][bb] is packed entry (min, max); walking bb, the
    // column-a part (bb < a) advances by nv - 1 - bb, the row-a part by 1
    // (two threads per row, each over half of bb and every component, were
    // measured no faster)
    for (int t = tid; t < dnv; t += NT) {
        const int c = t / nv, a = t - c * nv;
        const T* xc = xs + c * nv;
        const int offa = a * nv - a * (a - 1) / 2 - a;
        T acc = 0;
        int up = a;                                            // (bb, a), bb < a
        for (int bb = 0; bb < nv; ++bb) {
            const int idx = bb < a ? up : offa + bb;
            acc += Lp[idx] * xc[bb];
            up += nv - 1 - bb;
        }
        ys[t] = acc;
    }
    __syncthreads();
    for (int q = tid; q < np; q += NT) {
        T acc = 0;
        for (int x = 0; x < np; ++x) acc += Si[x * lds + q] * tq[x];
        sq[q] = acc;
    }
    __syncthreads();
    for (int a = tid; a < dnv; a += NT) {
        T z = ys[a];
        for (int q = 0; q < np; ++q) z += Wm[q * ldw + a] * sq[q];
        Y[s0 + a] = wq[a] * z;
    }
    for (int q = tid; q < np; q += NT) Y[s0 + dnv + q] = -wq[dnv + q] * sq[q];
}

__global__ void __launch_bounds__(SA_BULK_THREADS) saddle_apply_bulk_f32(
    int d, const int* __restrict__ poff, const int* __restrict__ pdofs, const int* __restrict__ pnv,
    const long long* __restrict__ foff, const float* __restrict__ fac, const float* __restrict__ r,
    const float* __restrict__ wt, float* __restrict__ Y, int buf_bytes, int xs_len, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_sb[];
    __shared__ __align__(8) unsigned long long bar;
    saddle_apply_bulk_body<float>(d, poff, pdofs, pnv, foff, fac, r, wt, Y, buf_bytes, xs_len, status, smem_sb, &bar);
}
__global__ void __launch_bounds__(SA_BULK_THREADS) saddle_apply_bulk_f64(
    int d, const int* __restrict__ poff, const int* __restrict__ pdofs, const int* __restrict__ pnv,
    const long long* __restrict__ foff, const double* __restrict__ fac, const double* __restrict__ r,
    const double* __restrict__ wt, double* __restrict__ Y, int buf_bytes, int xs_len, int* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem_sb[];
    __shared__ __align__(8) unsigned long long bar;
    saddle_apply_bulk_body<double>(d, poff, pdofs, pnv, foff, fac, r, wt, Y, buf_bytes, xs_len, status, smem_sb, &bar);
}

// ---------------------------------------------------------- coarse GJ ---
__global__ void __launch_bounds__(256) gj_step_pivot(int n, int k, double* __restrict__ A, int* __restrict__ ipiv,
                                                     double* __restrict__ colk, int* __restrict__ status) {
    __shared__ double s_val[8];
    __shared__ int s_idx[8];
    __shared__ int s_p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double best = -1.0;
    int bi = n;
    for (int i = k + tid; i < n; i += blockDim.x) {
        const double v = fabs(A[(long long)i * n + k]);
        if (v > best) { best = v; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = best; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (s_val[w] > best || (s_val[w] == best && s_idx[w] < bi)) { best = s_val[w]; bi = s_idx[w]; }
        if (!(best > 0.0) || bi >= n) { bi = k; if (*status == 0) *status = k + 1; }
        s_p = bi;
        ipiv[k] = bi;
    }
    __syncthreads();
    const int p = s_p;
    if (p != k)
        for (int j = tid; j < n; j += blockDim.x) {
            const double t = A[(long long)k * n + j];
            A[(long long)k * n + j] = A[(long long)p * n + j];
            A[(long long)p * n + j] = t;
        }
    __syncthreads();
    const double piv = A[(long long)k * n + k];
    const double inv = piv != 0.0 ? 1.0 / piv : 0.0;
    for (int i = tid; i < n; i += blockDim.x) colk[i] = A[(long long)i * n + k];
    __syncthreads();
    for (int j = tid; j < n; j += blockDim.x) A[(long long)k * n + j] = (j == k) ? inv : A[(long long)k * n + j] * inv;
}

__global__ void __launch_bounds__(256) gj_step_eliminate(int n, int k, double* __restrict__ A, const double* __restrict__ colk) {
    const long long total = (long long)n * n;
    const double inv = A[(long long)k * n + k];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t - (long long)i * n);
        if (i == k) continue;
        const double f = colk[i];
        if (j == k) A[t] = -f * inv;
        else A[t] -= f * A[(long long)k * n + j];
    }
}

// ---- blocked Gauss-Jordan inverse (partial pivoting) on every SM -------
// Panel [k0, k0 + B) of the row-major n x n matrix A: the columns of all rows
// in shared memory (pan[j n + i]), B Gauss-Jordan steps on them (pivot row
// p >= k with the largest |a_pk|, ties to the smaller row; swap; scale row k
// by r = 1 / a_kk and put r in place of a_kk; eliminate column k from every
// other row, putting -a_ik r in its place).  The panel columns go back to A
// and to Pk (row-major n x B) for the trailing update; ipiv[k] = p;
// status <- 1 + the step of the first zero pivot.
__global__ void __launch_bounds__(GJB_THREADS) gj_block_panel(int n, int k0, int B, double* __restrict__ A,
                                                              int* __restrict__ ipiv, double* __restrict__ Pk,
                                                              int* __restrict__ status) {
    extern __shared__ double pan[];
    __shared__ double rv[GJB_THREADS / 32];
    __shared__ int ri[GJB_THREADS / 32];
    __shared__ int s_p;
    __shared__ double s_r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    for (long long t = tid; t < (long long)n * B; t += nt) {
        const int i = (int)(t / B), j = (int)(t - (long long)i * B);
        pan[(long long)j * n + i] = A[(long long)i * n + k0 + j];
    }
    __syncthreads();
    for (int jj = 0; jj < B; ++jj) {
        const int k = k0 + jj;
        double* col = pan + (long long)jj * n;
        double best = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += nt) {
            const double v = fabs(col[i]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (lane == 0) { rv[warp] = best; ri[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nt / 32; ++w)
                if (rv[w] > best || (rv[w] == best && ri[w] < bi)) { best = rv[w]; bi = ri[w]; }
            if (!(best > 0.0) || bi >= n) {
                bi = k;
                if (*status == 0) *status = k + 1;
            }
            s_p = bi;
            ipiv[k] = bi;
            const double a = col[bi];
            s_r = a != 0.0 ? 1.0 / a : 0.0;
        }
        __syncthreads();
        const int p = s_p;
        const double r = s_r;
        for (int j = tid; j < B; j += nt) {
            double* cj = pan + (long long)j * n;
            if (p != k) { const double t = cj[k]; cj[k] = cj[p]; cj[p] = t; }
            cj[k] = j == jj ? r : cj[k] * r;
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            if (i == k) continue;
            const double f = col[i];
            for (int j = 0; j < B; ++j) {
                if (j == jj) continue;
                double* cj = pan + (long long)j * n;
                cj[i] = fma(-f, cj[k], cj[i]);
            }
            col[i] = -f * r;
        }
        __syncthreads();
    }
    for (long long t = tid; t < (long long)n * B; t += nt) {
        const int i = (int)(t / B), j = (int)(t - (long long)i * B);
        const double v = pan[(long long)j * n + i];
        A[(long long)i * n + k0 + j] = v;
        Pk[t] = v;
    }
}

// The same panel held by one thread-block cluster of GJC_CTAS CTAs: CTA r
// keeps rows [r R, (r + 1) R) of the panel's B columns in shared memory, in
// two buffers that alternate by pivot step, so one cluster barrier per pivot
// suffices: a step reads the current buffer (its own and, through distributed
// shared memory, the pivot row and the old row k of their owners) and writes
// the other, which nobody reads before the next barrier.  A step:
//   own candidate (largest |a_ik| over own rows i >= k; ties to the smaller
//   row) -> cluster barrier -> the 16 candidates read, pivot p chosen alike
//   everywhere -> pivot row (scaled by 1 / a_pk) and, in the CTA owning p,
//   the old row k read -> own rows eliminated into the other buffer.
// The per-pivot work is R B; the trailing columns are left to gj_block_swap
// / gj_block_update on every SM.
__global__ void __launch_bounds__(GJC_THREADS) gj_cluster_panel(int n, int k0, int B, double* __restrict__ A,
                                                                int* __restrict__ ipiv, double* __restrict__ Pk,
                                                                int* __restrict__ status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ double gsm[];
    const int R = (n + GJC_CTAS - 1) / GJC_CTAS;
    const int rank = (int)cluster.block_rank();
    const int r0 = rank * R, nr = max(0, min(R, n - r0));
    double* buf0 = gsm;                          // [R][B] rows, even steps read this one
    double* buf1 = buf0 + (size_t)R * B;         // [R][B] odd steps read this one
    double* prow = buf1 + (size_t)R * B;         // [B] scaled pivot row
    double* rowk = prow + B;                     // [B] old row k (CTA that owns p)
    __shared__ double cand_v[GJC_THREADS / 32], s_inv, s_cv[2], s_sv[2];
    __shared__ int cand_i[GJC_THREADS / 32], s_p, s_ci[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    for (int t = tid; t < nr * B; t += nt) {
        const int ii = t / B, j = t - ii * B;
        buf0[t] = A[(long long)(r0 + ii) * n + k0 + j];
    }
    __syncthreads();
    for (int jj = 0; jj < B; ++jj) {
        const int k = k0 + jj, par = jj & 1;
        double* cur = par ? buf1 : buf0;
        double* nxt = par ? buf0 : buf1;
        double bv = -1.0;
        int bi = n;
        for (int ii = tid; ii < nr; ii += nt) {
            const int i = r0 + ii;
            if (i < k) continue;
            const double av = fabs(cur[(size_t)ii * B + jj]);
            if (av > bv) { bv = av; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, bv, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (lane == 0) { cand_v[warp] = bv; cand_i[warp] = bi; }
        __syncthreads();
        if (warp == 0) {
            double b = lane < nt / 32 ? cand_v[lane] : -1.0;
            int i0 = lane < nt / 32 ? cand_i[lane] : n;
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, b, o);
                const int oi = __shfl_down_sync(0xffffffffu, i0, o);
                if (ob > b || (ob == b && oi < i0)) { b = ob; i0 = oi; }
            }
            if (lane == 0) {
                s_cv[par] = b;
                s_ci[par] = i0;
                s_sv[par] = i0 < n ? cur[(size_t)(i0 - r0) * B + jj] : 0.0;
            }
        }
        cluster.sync();                                            // candidates and rows of this step visible
        if (warp == 0) {
            double b = -1.0, sgn = 0.0;
            int p = n;
            if (lane < GJC_CTAS) {
                b = *cluster.map_shared_rank(&s_cv[par], lane);
                p = *cluster.map_shared_rank(&s_ci[par], lane);
                sgn = *cluster.map_shared_rank(&s_sv[par], lane);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, b, o), os = __shfl_down_sync(0xffffffffu, sgn, o);
                const int op = __shfl_down_sync(0xffffffffu, p, o);
                if (ob > b || (ob == b && op < p)) { b = ob; p = op; sgn = os; }
            }
            if (lane == 0) {
                if (!(b > 0.0) || p >= n) {
                    p = k;
                    sgn = 0.0;
                    if (rank == 0 && *status == 0) *status = k + 1;
                }
                s_p = p;
                s_inv = sgn != 0.0 ? 1.0 / sgn : 0.0;
                if (rank == 0) ipiv[k] = p;
            }
        }
        __syncthreads();
        const int p = s_p;
        const double inv = s_inv;
        {
            const double* src = cluster.map_shared_rank(cur, p / R) + (size_t)(p % R) * B;
            for (int j = tid; j < B; j += nt) prow[j] = j == jj ? inv : src[j] * inv;
            if (p != k && p >= r0 && p < r0 + nr) {
                const double* srk = cluster.map_shared_rank(cur, k / R) + (size_t)(k % R) * B;
                for (int j = tid; j < B; j += nt) rowk[j] = srk[j];
            }
        }
        __syncthreads();
        // (cur is only read in this step, so each thread takes its row's
        // multiplier from it directly)
        for (int t = tid; t < nr * B; t += nt) {
            const int ii = t / B, j = t - ii * B;
            const int i = r0 + ii;
            if (i == k) {
                nxt[t] = prow[j];
            } else {
                const double f = i == p ? rowk[jj] : cur[(size_t)ii * B + jj];
                const double src = i == p ? rowk[j] : cur[t];
                nxt[t] = j == jj ? -f * inv : fma(-f, prow[j], src);
            }
        }
        __syncthreads();
    }
    // every CTA must be done reading the others' buffers before any exits
    cluster.sync();
    const double* fin = (B & 1) ? buf1 : buf0;
    for (int t = tid; t < nr * B; t += nt) {
        const int ii = t / B, j = t - ii * B;
        A[(long long)(r0 + ii) * n + k0 + j] = fin[t];
        Pk[(long long)(r0 + ii) * B + j] = fin[t];
    }
}

// The panel's row swaps on every column outside it, and the swapped rows
// k0 .. k0 + B - 1 copied to Yb[j n + c] (before the update overwrites them).
__global__ void __launch_bounds__(256) gj_block_swap(int n, int k0, int B, double* __restrict__ A,
                                                     const int* __restrict__ ipiv, double* __restrict__ Yb) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n || (c >= k0 && c < k0 + B)) return;
    for (int jj = 0; jj < B; ++jj) {
        const int k = k0 + jj, p = ipiv[k];
        if (p != k) {
            const double t = A[(long long)k * n + c];
            A[(long long)k * n + c] = A[(long long)p * n + c];
            A[(long long)p * n + c] = t;
        }
    }
    for (int jj = 0; jj < B; ++jj) Yb[(long long)jj * n + c] = A[(long long)(k0 + jj) * n + c];
}

// Trailing update of the columns outside the panel, on 32 x 32 tiles:
//   A[i][c] = (i in panel rows ? 0 : A[i][c]) + sum_j Pk[i][j] Yb[j][c].
__global__ void __launch_bounds__(256) gj_block_update(int n, int k0, int B, double* __restrict__ A,
                                                       const double* __restrict__ Pk, const double* __restrict__ Yb) {
    __shared__ double ys[GJB_MAX_B][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane, i0 = blockIdx.y * 32;
    const bool colok = c < n && !(c >= k0 && c < k0 + B);
    for (int jj = warp; jj < B; jj += 8) ys[jj][lane] = colok ? Yb[(long long)jj * n + c] : 0.0;
    __syncthreads();
    if (!colok) return;
    for (int i = i0 + warp; i < min(n, i0 + 32); i += 8) {
        const double* pk = Pk + (long long)i * B;
        double acc = (i >= k0 && i < k0 + B) ? 0.0 : A[(long long)i * n + c];
        for (int jj = 0; jj < B; ++jj) acc = fma(pk[jj], ys[jj][lane], acc);
        A[(long long)i * n + c] = acc;
    }
}

__global__ void gj_unpivot_rows(int n, double* __restrict__ A, const int* __restrict__ ipiv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int k = n - 1; k >= 0; --k) {
            const int p = ipiv[k];
            if (p != k) {
                const double t = A[(long long)i * n + k];
                A[(long long)i * n + k] = A[(long long)i * n + p];
                A[(long long)i * n + p] = t;
            }
        }
}

// ------------------------------------------------------ small Hessenberg ---
__global__ void fgmres_givens(int j, int ldh, double* __restrict__ H, const double* __restrict__ hcol,
                              const double* __restrict__ hnorm, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ resid) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) H[i * ldh + j] = hcol[i];
    H[(j + 1) * ldh + j] = hnorm[0];
    for (int i = 0; i < j; ++i) {
        const double a = H[i * ldh + j], b = H[(i + 1) * ldh + j];
        H[i * ldh + j] = cs[i] * a + sn[i] * b;
        H[(i + 1) * ldh + j] = -sn[i] * a + cs[i] * b;
    }
    const double a = H[j * ldh + j], b = H[(j + 1) * ldh + j];
    const double den = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (den > 0.0) { c = a / den; s = b / den; }
    cs[j] = c;
    sn[j] = s;
    H[j * ldh + j] = den > 0.0 ? den : a;
    H[(j + 1) * ldh + j] = 0.0;
    g[j + 1] = -s * g[j];
    g[j] = c * g[j];
    resid[0] = fabs(g[j + 1]);
}

__global__ void fgmres_backsolve(int m, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                                 double* __restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = m - 1; i >= 0; --i) {
        double s = g[i];
        for (int l = i + 1; l < m; ++l) s -= H[i * ldh + l] * y[l];
        y[i] = s / H[i * ldh + i];
    }
}

__global__ void arnoldi_store(int j, int m, double* __restrict__ Hs, const double* __restrict__ h,
                              const double* __restrict__ hnorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int i = 0; i <= j; ++i) Hs[i * m + j] = h[i];
    Hs[(j + 1) * m + j] = hnorm[0];
}


__host__ __device__ inline cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cplx cmul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline cplx cconj(cplx a) { return {a.re, -a.im}; }
__host__ __device__ inline double cabs2(cplx a) { return hypot(a.re, a.im); }
__host__ __device__ inline cplx csqrt2(cplx z) {
    const double r = cabs2(z);
    double re = sqrt(fmax(0.0, 0.5 * (r + z.re)));
    double im = sqrt(fmax(0.0, 0.5 * (r - z.re)));
    if (z.im < 0) im = -im;
    return {re, im};
}
__host__ __device__ inline cplx cscale(cplx a, double s) { return {a.re * s, a.im * s}; }

// Eigenvalues of a small upper Hessenberg matrix by the shifted QR
// iteration in complex arithmetic (Wilkinson shift from the trailing 2 x 2
// block, Givens rotations, deflation on negligible subdiagonals).  Writes
// out[0] = largest real part, out[1] = 0 if converged, 1 otherwise.
__host__ __device__ void hessenberg_eig_core(int m, int ld, const double* Hs, double* out, cplx (*A)[HESS_MAX],
                                             cplx* cr, cplx* sr) {
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) A[i][j] = {(j >= i - 1) ? Hs[i * ld + j] : 0.0, 0.0};
    double best = -1e300;
    int hi = m - 1, it = 0, total = 0, failed = 0;
    while (hi >= 0) {
        if (hi == 0) { best = fmax(best, A[0][0].re); break; }
        int l = hi;
        while (l > 0) {
            const double sub = cabs2(A[l][l - 1]);
            const double diag = cabs2(A[l][l]) + cabs2(A[l - 1][l - 1]);
            if (sub <= 1e-15 * (diag > 0 ? diag : 1.0)) break;
            --l;
        }
        if (l == hi) { best = fmax(best, A[hi][hi].re); --hi; it = 0; continue; }
        if (++total > 200 * m) { failed = 1; for (int i = 0; i <= hi; ++i) best = fmax(best, A[i][i].re); break; }
        const cplx a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
        const cplx half = cscale(csub(a, d), 0.5);
        const cplx disc = csqrt2(cadd(cmul(half, half), cmul(b, c)));
        const cplx mid = cscale(cadd(a, d), 0.5);
        const cplx m1 = cadd(mid, disc), m2 = csub(mid, disc);
        cplx mu = cabs2(csub(m1, d)) < cabs2(csub(m2, d)) ? m1 : m2;
        if (++it % 11 == 10) mu = cadd(d, cplx{cabs2(c), 0.0});   // exceptional shift
        for (int i = l; i <= hi; ++i) A[i][i] = csub(A[i][i], mu);
        for (int i = l; i < hi; ++i) {
            const cplx x = A[i][i], y = A[i + 1][i];
            const double r = hypot(cabs2(x), cabs2(y));
            cplx cc = {1.0, 0.0}, ss = {0.0, 0.0};
            if (r > 0) { cc = cscale(x, 1.0 / r); ss = cscale(y, 1.0 / r); }
            cr[i] = cc;
            sr[i] = ss;
            for (int j = i; j <= hi; ++j) {
                const cplx u = A[i][j], v = A[i + 1][j];
                A[i][j] = cadd(cmul(cconj(cc), u), cmul(cconj(ss), v));
                A[i + 1][j] = csub(cmul(cc, v), cmul(ss, u));
            }
        }
        for (int i = l; i < hi; ++i) {
            const cplx cc = cr[i], ss = sr[i];
            const int rmax = (i + 2 < hi) ? i + 2 : hi;
            for (int rr = l; rr <= rmax; ++rr) {
                const cplx u = A[rr][i], v = A[rr][i + 1];
                A[rr][i] = cadd(cmul(u, cc), cmul(v, ss));
                A[rr][i + 1] = csub(cmul(v, cconj(cc)), cmul(u, cconj(ss)));
            }
        }
        for (int i = l; i <= hi; ++i) A[i][i] = cadd(A[i][i], mu);
    }
    out[0] = best;
    out[1] = failed;
}

__global__ void __launch_bounds__(256) fp64_fma_probe(long long iters, double a, double b, double never,
                                                      double* __restrict__ out) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = 1e-3 * (threadIdx.x + 1) + u;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = fma(x[u], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == never) out[blockIdx.x] = s;
}

}  // namespace skern
