// sm_103a kernels of the phMG hot path.
//
//   spmv_*            CSR SpMV / fused residual r = b - K x (Eq. 3.1, 3.2
//                     residuals), prolongation y += P x and restriction y = R x
//                     (Sec. 3.1 transfers).
//   patch_gather      K_i = I_i K I_i^T from the CSR operator (Eq. 3.4,
//                     Sec. 3.4 assembled-matrix patch extraction).
//   gj_inverse_*      batched partial-pivot Gauss-Jordan inversion of the
//                     patch matrices in FP64 (exact patch solves, Sec. 3.4).
//   patch_apply       y_i = W_i K_i^{-1} (I_i r) for every patch (one ASM
//                     sweep, Eq. 3.4), streamed from HBM.
//   pull_scatter      z = sum_i I_i^T y_i as a deterministic gather over the
//                     DoF -> (patch slot) transpose map, fused with the
//                     Chebyshev / damped update.
//   mdot / maxpy ...  FGMRES and Arnoldi vector kernels (FP64).
//   hess_*            small Hessenberg / Givens kernels run by one thread.
//
// All kernels take plain device pointers; grids are sized by the host.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace skern {

constexpr int GJ_SMEM_MAX_N = 160;   // FP64 patch held in shared memory up to this size

// Programmatic dependent launch: a kernel launched with the programmatic
// stream serialisation attribute may start while the kernel before it on the
// stream is still running.  pdl_wait() blocks until that kernel has finished
// and its writes are visible; every kernel of the V-cycle calls it before it
// reads an input another kernel writes, or writes anything, and may read
// constant data (operators, patch factors, maps) before it.  pdl_release()
// lets the next kernel's blocks be scheduled once every block of this one has
// called it or exited.  Both are no-ops in a kernel launched without the
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ----------------------------------------------------------------- SpMV ---
enum SpmvMode { SPMV_SET = 0, SPMV_ADD = 1, SPMV_RESID = 2 };

// One LANES-wide group of threads per row; values of type T accumulate in T.
// mode SET:   y = A x        ADD: y += A x        RESID: y = b - A x
template <typename T, int LANES, int MODE>
__global__ void __launch_bounds__(256) spmv_csr(int nrows, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const T* __restrict__ av, const T* __restrict__ x,
                                                T* __restrict__ y, const T* __restrict__ b) {
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int row = gtid / LANES;
    const int lane = threadIdx.x % LANES;
    // the operator is constant: its first round of column and value loads
    // is issued before waiting for the kernel that wrote x (and b)
    const bool live = row < nrows;
    const int s = live ? __ldg(rp + row) : 0, e = live ? __ldg(rp + row + 1) : 0;
    int c[4];
    T a[4];
    int base = s + lane;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int p = base + u * LANES;
        const bool ok = p < e;
        c[u] = ok ? __ldg(ci + p) : 0;
        a[u] = ok ? __ldg(av + p) : T(0);
    }
    pdl_wait();
    pdl_release();
    if (!live) return;   // whole LANES-group exits together (LANES divides 32)
    T acc = 0;
    // four entries per lane per round: their column and value loads, then
    // their x loads, are issued together (a row of ~40 entries takes one
    // round at 16 lanes instead of a chain of three dependent load pairs)
    for (;;) {
#pragma unroll
        for (int u = 0; u < 4; ++u) acc += a[u] * x[c[u]];
        base += 4 * LANES;
        if (base >= e) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = base + u * LANES;
            const bool ok = p < e;
            c[u] = ok ? __ldg(ci + p) : 0;
            a[u] = ok ? __ldg(av + p) : T(0);
        }
    }
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, LANES);
    if (lane == 0) {
        if (MODE == SPMV_SET) y[row] = acc;
        else if (MODE == SPMV_ADD) y[row] += acc;
        else y[row] = b[row] - acc;
    }
}

// ------------------------------------------------------- vector kernels ---
template <typename TO, typename TI>
__global__ void convert_vec(int n, const TI* __restrict__ x, TO* __restrict__ y) {
    pdl_wait();
    pdl_release();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = (TO)x[i];
}

template <typename T>
__global__ void fill_vec(long long n, T v, T* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) y[i] = v;
}

// y = a x + b y
template <typename T>
__global__ void axpby(int n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
    pdl_wait();
    pdl_release();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] = a * x[i] + b * y[i];
}

// y = x * (1 / *s)   (device scalar divisor, FGMRES / Arnoldi normalisation)
__global__ void scale_by_inv(int n, const double* __restrict__ x, const double* __restrict__ s, double* __restrict__ y);

// y = x - K x is not needed; the FGMRES/Arnoldi reductions:
// partial[b*m + i] = sum over this block's rows of V[i][k] * w[k]
__global__ void mdot_partial(int n, int m, const double* __restrict__ V, long long ldv,
                             const double* __restrict__ w, double* __restrict__ partial);
// out[i] = sum_b partial[b*m + i] (fixed order), optionally accumulated
// into acc[i] as well; if sqrt_out, out[0] = sqrt(sum).
__global__ void mdot_final(int nblocks, int m, const double* __restrict__ partial, double* __restrict__ out,
                           double* __restrict__ acc, int sqrt_out);
// Same reduction in one launch (last block finishes in a fixed order);
// MDOT_BLOCKS blocks of MDOT_THREADS threads; ticket must start at 0 and is reset.
constexpr int MDOT_BLOCKS = 152, MDOT_THREADS = 256;
void mdot_fused(int n, int m, const double* V, long long ldv, const double* w, double* partial, unsigned int* ticket,
                double* out, double* acc, int sqrt_out, cudaStream_t s);
// w <- w - V h; out[0..m) = V^T w, out[m] = w^T w of the updated w,
// acc[i] += out[i] (i < m); MDOT_BLOCKS blocks of MDOT_THREADS threads, m <= 31.
void maxpy_mdot(int n, int m, const double* V, long long ldv, const double* h, double* w, double* partial,
                unsigned int* ticket, double* out, double* acc, cudaStream_t s);
// w <- (w - V h) / nu, nu = sqrt(max(*nrm2 - |h|^2, 0)), *hn = nu
__global__ void maxpy_normalise(int n, int m, const double* __restrict__ V, long long ldv, const double* __restrict__ h,
                                const double* __restrict__ nrm2, double* __restrict__ w, double* __restrict__ hn);
// w[k] += sign * sum_i h[i] V[i][k]
__global__ void maxpy(int n, int m, const double* __restrict__ V, long long ldv, const double* __restrict__ h,
                      double sign, double* __restrict__ w);

// ------------------------------------------------------ DoF -> slot map ---
// slot_count (cnt zeroed) -> exclusive scan of cnt into soff[0..n] ->
// slot_fill (cur zeroed) -> slot_sort: sidx lists every DoF's slots in
// increasing order, wt[j] = 1 / multiplicity.
__global__ void slot_count(long long nent, const int* __restrict__ pdofs, int* __restrict__ cnt);
__global__ void slot_fill(long long nent, const int* __restrict__ pdofs, const int* __restrict__ soff, int* __restrict__ cur,
                          int* __restrict__ sidx);
__global__ void slot_sort(int n, const int* __restrict__ soff, int* __restrict__ sidx, double* __restrict__ wt);

// ------------------------------------------------------------- patches ---
// Dense K_i (row-major n_i x n_i, FP64) gathered from the CSR of K: one CTA
// per patch; column positions found by binary search in the sorted patch DoF
// list.  out must be zeroed by the caller.
__global__ void patch_gather(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                             const long long* __restrict__ moff, const int* __restrict__ rp,
                             const int* __restrict__ ci, const double* __restrict__ av, double* __restrict__ out);

// In-place Gauss-Jordan inversion with partial pivoting of every patch
// matrix (row-major, FP64), shared-memory variant (n_i <= GJ_SMEM_MAX_N).
// Writes K_i^{-1} column-major with leading dimension ld64 (FP64) and, if
// inv32 != nullptr, ld32 (FP32); the row-major inverse is also written back
// to `work` when keep_rowmajor.  status[patch] = 0, or 1 + pivot step of the
// first zero pivot.
__global__ void gj_inverse_smem(int npatch, const int* __restrict__ poff, const long long* __restrict__ moff,
                                double* __restrict__ work, const long long* __restrict__ off64, double* __restrict__ inv64,
                                const long long* __restrict__ off32, float* __restrict__ inv32,
                                int* __restrict__ status, int only_large);
// Same algorithm operating on the matrix in global memory (large patches).
__global__ void gj_inverse_global(int npatch, const int* __restrict__ poff, const long long* __restrict__ moff,
                                  double* __restrict__ work, const long long* __restrict__ off64, double* __restrict__ inv64,
                                  const long long* __restrict__ off32, float* __restrict__ inv32,
                                  int* __restrict__ status, int* __restrict__ ipiv_ws, double* __restrict__ col_ws);

// Block (Schur-complement) inverse of saddle-structured Vanka patches:
// K_i = [L 0 B_0^T; 0 L B_1^T; B_0 B_1 0] with one SPD velocity block L per
// component (vector Laplacian), pnv[p] velocity nodes per component.  FP64;
// SPD blocks inverted by Gauss-Jordan without pivoting; status as above.
// Patches whose scratch (saddle_scratch doubles) is <= max_scratch run in
// shared memory (saddle_inverse_smem), the others in the global scratch at
// soff[p] (saddle_inverse_global).
__host__ __device__ inline long long saddle_scratch(int d, int n, int nv) {
    const int np = n - d * nv, npp = np | 1;
    const int mx = nv > np ? nv : np;
    return (long long)nv * nv + 2LL * d * nv * npp + (long long)np * np + 3LL * mx + 2;
}
constexpr long long SADDLE_SMEM_MAX_DOUBLES = 25600;   // 200 KB of shared memory
// scratch of the factored-only inversion (one component's B^T and W at a
// time, the two-pivot sweep's columns, and one bit mask per pressure column
// of B^T: its nonzero rows)
// Pair-packed upper triangle of a symmetric n x n matrix: rows pr and
// n - 1 - pr share the n + 1 slots from pr (n + 1), in the order of the
// sweeps' row-pair mapping; entry (a, b), a <= b, sits at pp_row(n, a) + b.
__host__ __device__ inline long long pp_size(int n) { return (long long)((n + 1) / 2) * (n + 1); }
__host__ __device__ inline int pp_row(int n, int a) { return 2 * a < n ? a * n : (n - 1 - a) * (n + 1) + 1; }
// pp: the velocity block pair-packed (the shared-memory kernel) or full
// (the global-scratch kernel, whose lane accesses then stay coalesced)
__host__ __device__ inline long long saddle_scratch_factored(int d, int n, int nv, bool pp = true) {
    const int np = n - d * nv, npp = np | 1;
    const int mx = nv > np ? nv : np;
    return (pp ? pp_size(nv) : (long long)nv * nv) + 2LL * nv * npp + (long long)np * np + 7LL * mx + 2 + (long long)np * ((nv + 63) / 64);
}
// Outputs (each may be NULL): explicit inverses inv64 / inv32 (column-major,
// leading dimension n rounded up to 2 / 4), the factored form fac64 / fac32
// at foff64[p] / foff32[p] (saddle_factor_len), and, if back, the explicit
// inverse row-major in place of K_i.  saddle_inverse_smem with work == NULL
// (factored form only) reads each patch's rows of the CSR operator (rp, ci,
// av) directly, its sorted DoF list pdofs[poff[p] ..) held in shared memory
// at double offset sd_off (after the scratch).
__global__ void saddle_inverse_smem(int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pnv,
                                    const long long* __restrict__ moff, double* __restrict__ work,
                                    const long long* __restrict__ off64, double* __restrict__ inv64,
                                    const long long* __restrict__ off32, float* __restrict__ inv32,
                                    const long long* __restrict__ foff64, double* __restrict__ fac64,
                                    const long long* __restrict__ foff32, float* __restrict__ fac32, int back,
                                    int packed, long long max_scratch, const int* __restrict__ pdofs,
                                    const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
                                    int sd_off, int* __restrict__ status);
__global__ void saddle_inverse_global(int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pnv,
                                      const long long* __restrict__ moff, double* __restrict__ work,
                                      const long long* __restrict__ off64, double* __restrict__ inv64,
                                      const long long* __restrict__ off32, float* __restrict__ inv32,
                                      const long long* __restrict__ foff64, double* __restrict__ fac64,
                                      const long long* __restrict__ foff32, float* __restrict__ fac32, int back,
                                      int packed, long long max_scratch, const long long* __restrict__ soff,
                                      double* __restrict__ scratch, int* __restrict__ status);
// Elements of one patch's factored inverse (Li, W, Si with leading
// dimensions rounded up to vec = 2 (FP64) or 4 (FP32)); packed: Li as its
// upper triangle row by row (nv (nv + 1) / 2 entries, rounded up to vec),
// the layout of the bulk-copy apply.
__host__ __device__ inline long long saddle_factor_len(int d, int n, int nv, int vec, int packed = 0) {
    const int np = n - d * nv;
    const long long ldl = (nv + vec - 1) / vec * vec, ldw = (d * nv + vec - 1) / vec * vec,
                    lds = (np + vec - 1) / vec * vec;
    const long long lenL = packed ? ((long long)nv * (nv + 1) / 2 + vec - 1) / vec * vec : ldl * nv;
    return lenL + ldw * np + lds * np;
}
// Shared memory (bytes) of saddle_apply_*: partial sums, W (ws_len
// elements; 0 = W read from global memory), and five vectors of xs_len
// (>= the largest patch) elements.  W is staged when the total stays within
// SADDLE_APPLY_SMEM_MAX bytes (the kernels' shared-memory attribute).
constexpr int SADDLE_APPLY_THREADS = 128;
constexpr size_t SADDLE_APPLY_SMEM_MAX = 200 * 1024;
__host__ __device__ inline size_t saddle_apply_smem(int elem_bytes, int vec, long long ws_len, long long xs_len) {
    return (size_t)elem_bytes * vec * SADDLE_APPLY_THREADS * 3 + (size_t)elem_bytes * (ws_len + 5 * xs_len);
}
// The same sweep with one CTA per patch whose factored block is brought into
// shared memory by one bulk copy (buf_bytes >= the largest block, a
// multiple of 128; xs_len >= the largest patch).  *status = 1 if a CTA gave
// up waiting for its copy (bounded wait).
constexpr int SA_BULK_THREADS = 128;
constexpr long long SA_WAIT_LIMIT = 1ll << 22;
__host__ __device__ inline size_t saddle_apply_bulk_smem(int buf_bytes, int elem_bytes, int xs_len) {
    return (size_t)buf_bytes + (size_t)elem_bytes * 5 * xs_len;
}
__global__ void saddle_apply_bulk_f32(int d, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                      const int* __restrict__ pnv, const long long* __restrict__ foff,
                                      const float* __restrict__ fac, const float* __restrict__ r,
                                      const float* __restrict__ wt, float* __restrict__ Y, int buf_bytes,
                                      int xs_len, int* __restrict__ status);
__global__ void saddle_apply_bulk_f64(int d, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                      const int* __restrict__ pnv, const long long* __restrict__ foff,
                                      const double* __restrict__ fac, const double* __restrict__ r,
                                      const double* __restrict__ wt, double* __restrict__ Y, int buf_bytes,
                                      int xs_len, int* __restrict__ status);
__global__ void saddle_apply_f32(int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                 const int* __restrict__ pnv, const long long* __restrict__ foff,
                                 const float* __restrict__ fac, const float* __restrict__ r, const float* __restrict__ wt,
                                 float* __restrict__ Y, int xs_len, int ws_len);
__global__ void saddle_apply_f64(int npatch, int d, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                 const int* __restrict__ pnv, const long long* __restrict__ foff,
                                 const double* __restrict__ fac, const double* __restrict__ r,
                                 const double* __restrict__ wt, double* __restrict__ Y, int xs_len, int ws_len);

// One ASM sweep (Eq. 3.4): Y[poff[i] + a] = w[dof_a] * sum_b Kinv_i[a][b] r[dof_b].
// FP32: float4 loads of 4 consecutive rows per thread; FP64: double2 loads
// of 2 rows.  One CTA per patch; blockDim = round_up(ld / VEC, 32).
__global__ void patch_apply_f32(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                const long long* __restrict__ ioff, const float* __restrict__ inv,
                                const float* __restrict__ r, const float* __restrict__ wt, float* __restrict__ Y);
__global__ void patch_apply_f64(int npatch, const int* __restrict__ poff, const int* __restrict__ pdofs,
                                const long long* __restrict__ ioff, const double* __restrict__ inv,
                                const double* __restrict__ r, const double* __restrict__ wt, double* __restrict__ Y);

// out[j] = alpha * sum_{s in slots(j)} Y[s] + beta * out[j]  (slots in a
// fixed order, so the sum is bitwise reproducible).  Fused Chebyshev
// bookkeeping: xmode PULL_X_SET also sets x[j] = out[j], PULL_X_ADD adds
// x[j] += out[j]; with rdst != NULL, rdst[j] = bsrc[j].
enum PullX { PULL_X_NONE = 0, PULL_X_SET = 1, PULL_X_ADD = 2 };
template <typename T>
__global__ void __launch_bounds__(256) pull_scatter(int n, const int* __restrict__ soff, const int* __restrict__ sidx,
                                                    const T* __restrict__ Y, T alpha, T beta, T* __restrict__ out,
                                                    T* __restrict__ x, int xmode, const T* __restrict__ bsrc,
                                                    T* __restrict__ rdst) {
    pdl_wait();
    pdl_release();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        T s = 0;
        const int e = soff[j + 1];
        for (int q = soff[j]; q < e; ++q) s += Y[sidx[q]];
        const T o = beta == T(0) ? alpha * s : alpha * s + beta * out[j];
        out[j] = o;
        if (xmode == PULL_X_SET) x[j] = o;
        else if (xmode == PULL_X_ADD) x[j] += o;
        if (rdst) rdst[j] = bsrc[j];
    }
}

// ------------------------------------------------------ coarse solve ---
// One Gauss-Jordan step k on a dense row-major n x n FP64 matrix in global
// memory: pivot search, row swap, pivot-row scaling and copy of column k
// (single CTA), then the rank-1 elimination over all rows (whole grid).
__global__ void gj_step_pivot(int n, int k, double* __restrict__ A, int* __restrict__ ipiv,
                              double* __restrict__ colk, int* __restrict__ status);
__global__ void gj_step_eliminate(int n, int k, double* __restrict__ A, const double* __restrict__ colk);
__global__ void gj_unpivot_rows(int n, double* __restrict__ A, const int* __restrict__ ipiv);
// Blocked Gauss-Jordan inverse of one n x n row-major matrix on every SM,
// B <= GJB_MAX_B pivots per panel: for each panel gj_block_panel (one CTA,
// gj_block_panel_smem bytes), gj_block_swap (one thread per column),
// gj_block_update (grid ceil(n/32) x ceil(n/32)); then gj_unpivot_rows.
constexpr int GJB_THREADS = 512, GJB_MAX_B = 32;
__host__ __device__ inline size_t gj_block_panel_smem(int n, int B) { return (size_t)n * B * sizeof(double); }
__global__ void gj_block_panel(int n, int k0, int B, double* __restrict__ A, int* __restrict__ ipiv,
                               double* __restrict__ Pk, int* __restrict__ status);
__global__ void gj_block_swap(int n, int k0, int B, double* __restrict__ A, const int* __restrict__ ipiv,
                              double* __restrict__ Yb);
__global__ void gj_block_update(int n, int k0, int B, double* __restrict__ A, const double* __restrict__ Pk,
                                const double* __restrict__ Yb);
constexpr int GJC_CTAS = 16, GJC_THREADS = 512;
// The panel on one cluster of GJC_CTAS CTAs (rows split among them):
// gj_cluster_panel_smem_doubles(n, B) doubles of dynamic shared memory.
__host__ __device__ inline long long gj_cluster_panel_smem_doubles(int n, int B) {
    const long long R = (n + GJC_CTAS - 1) / GJC_CTAS;
    return 2 * R * B + 2LL * B + R;
}
__global__ void gj_cluster_panel(int n, int k0, int B, double* __restrict__ A, int* __restrict__ ipiv,
                                 double* __restrict__ Pk, int* __restrict__ status);


// y[i] = sum_j A[i][j] x[j] for i < nout (row-major, leading dimension lda),
// one warp per row, accumulated in FP64 whatever the vectors' type (an FP32
// x is widened exactly, y rounded once)
template <typename TI, typename TO>
__global__ void __launch_bounds__(256) dense_gemv(int nout, int ncol, int lda, const double* __restrict__ A,
                                                  const TI* __restrict__ x, TO* __restrict__ y) {
    pdl_wait();
    pdl_release();
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= nout) return;
    double s = 0;
    for (int j = lane; j < ncol; j += 32) s += A[(long long)row * lda + j] * (double)x[j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = (TO)s;
}

// --------------------------------------------------- small Hessenberg ---
// FGMRES: apply the previous Givens rotations to column j of H (stored
// [restart+1][restart] row-major), build rotation j, update g; resid[0] = |g[j+1]|.
// hcol holds h[0..j]; hnorm[0] = h[j+1].
__global__ void fgmres_givens(int j, int ldh, double* __restrict__ H, const double* __restrict__ hcol,
                              const double* __restrict__ hnorm, double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, double* __restrict__ resid);
// y = H[0:m,0:m]^{-1} g (upper triangular back substitution)
__global__ void fgmres_backsolve(int m, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                                 double* __restrict__ y);
// Arnoldi: store column j of H (h[0..j], hnorm) into Hs [(m+1) x m].
__global__ void arnoldi_store(int j, int m, double* __restrict__ Hs, const double* __restrict__ h,
                              const double* __restrict__ hnorm);
constexpr int HESS_MAX = 16;
struct cplx { double re, im; };
__host__ __device__ void hessenberg_eig_core(int m, int ld, const double* Hs, double* out, cplx (*A)[HESS_MAX],
                                             cplx* cr, cplx* sr);
// Eigenvalues of the leading m x m block of an upper Hessenberg matrix
// (row-major, leading dimension ld) by the shifted QR iteration in complex
// arithmetic; out[0] = largest real part, out[1] = 1 if not converged.
// Host and device callable; the library runs it on the host.
// ------------------------------------------------------ solve plumbing ---
// b_free[r] = (F restricted) computed by the host-built maps:
// x_free gathers: out[i] = in[idx[i]]; scatter: out[idx[i]] = in[i]
template <typename T>
__global__ void gather_idx(int n, const int* __restrict__ idx, const T* __restrict__ in, T* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = in[idx[i]];
}
template <typename T>
__global__ void scatter_idx(int n, const int* __restrict__ idx, const T* __restrict__ in, T* __restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[idx[i]] = in[i];
}
// x[i] -= mean; mean = (sum_i w[i] x[i]) / wsum from a device scalar
__global__ void sub_scalar(int n, double* __restrict__ x, const double* __restrict__ num, double den);
// z[qcell[e][a]] = scale[e] * sum_b minv[a][b] y[qcell[e][b]]: a block-diagonal
// operator whose blocks are one reference matrix times a per-cell scale (the
// cells own disjoint index sets)
__global__ void block_mass_inverse(int nc, int nb, const int* __restrict__ qcell, const double* __restrict__ minv,
                                   const double* __restrict__ scale, const double* __restrict__ y, double* __restrict__ z);
// rows [0, nr), columns [0, nc) of a CSR: per-row counts, then (after a scan
// into brp) the entries in their row order, FP64 and optionally FP32
__global__ void csr_block_count(int nr, int nc, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ len);
__global__ void csr_block_fill(int nr, int nc, const int* __restrict__ rp, const int* __restrict__ ci,
                               const double* __restrict__ v, const int* __restrict__ brp, int* __restrict__ bci,
                               double* __restrict__ bv, float* __restrict__ bv32);
// x[i] -= w[i] * num[0] / den
// FP64 pipe peak probe: every thread runs 8 independent FMA chains of
// `iters` steps (x = x * a + b); out is written only if the sum equals the
// impossible value `never`, which keeps the chains live.
__global__ void fp64_fma_probe(long long iters, double a, double b, double never, double* __restrict__ out);

__global__ void sub_weighted(int n, double* __restrict__ x, const double* __restrict__ w, const double* __restrict__ num,
                             double den);

}  // namespace skern
