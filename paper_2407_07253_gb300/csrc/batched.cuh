// Kernels of the batched (multi-right-hand-side) V-cycle.
//
// The m right-hand sides of one batch are interleaved DoF-major: vector v of
// a level is stored as X[j * m + c] (DoF j, right-hand side c), m a multiple
// of 8.  A sparse matrix is then read once per batch, every gathered row is
// m contiguous floats, and the patch apply becomes one dense GEMM per patch,
//   Y_i (n_i x m) = W_i K_i^{-1} (n_i x n_i) R_i (n_i x m),
// which runs on the tensor cores (warp-level m16n8k8 TF32 MMA; the 3xTF32
// split a = a_hi + a_lo keeps FP32 accuracy).  At m = 64 the GEMM does
// 2 m = 128 flop per 4-byte inverse entry, so it is bound by streaming the
// FP32 inverses from HBM, not by the MMA rate.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace sbat {

enum GemmMode { GEMM_TF32 = 0, GEMM_3XTF32 = 1 };

// X[j * m + c] = (float) r[c * n + j] for c < nrhs, 0 for nrhs <= c < m
void to_interleaved(int n, int nrhs, int m, const double* r, float* X, cudaStream_t s);
// z[c * n + j] = X[j * m + c] for c < nrhs
void from_interleaved(int n, int nrhs, int m, const float* X, double* z, cudaStream_t s);

// Y = A X (mode 0), Y += A X (mode 1), Y = B - A X (mode 2); A in CSR (FP32
// values), X, Y, B interleaved with width m.
void spmm(int mode, int nr, int m, const int* rp, const int* ci, const float* av, const float* X, float* Y,
          const float* B, cudaStream_t s);

// nullptr if patch_gemm of this mode and width handles patches of <= maxn
// DoFs on the current device, else the reason (shared or tensor memory)
const char* patch_gemm_check(int mode, int maxn, int m);

// self-test of the tensor-core kernel's bounded mbarrier wait (writes 2 to
// *result_dev when a wait on a barrier nobody arrives on gives up and the
// kernel returns); returns the launch's cudaError_t
int wait_probe(long long polls, int* result_dev, cudaStream_t s);

// bytes of the per-patch tensor maps of a level, and their construction
// (host encoding from the device offsets; synchronous)
size_t tmap_bytes(int npatch);
void build_tmaps(int npatch, const int* poff, const long long* ioff, const float* inv, void* tmaps);

// Yb[(poff[p] + a) * m + c] = wt[dof] * (K_p^{-1} R_p)[a][c], R_p[a][c] =
// X[pdofs[poff[p] + a] * m + c], for the nlist patches p = plist[i] (plist
// NULL: p = i < nlist); inverses column-major with leading dimension
// (n + 3) & ~3 at ioff[p] (the FP32 ASM layout), symmetric.
//   kind GEMM_KIND_TC     tcgen05 tensor cores; GEMM_TF32 reads the inverses
//                         through tmaps (build_tmaps over inv), GEMM_3XTF32
//                         through tmaps_hi / tmaps_lo (build_tmaps over the
//                         split_tf32 parts, same layout) with three MMAs per
//                         k-step;
//   kind GEMM_KIND_WARP   warp-level MMA, nw warps per CTA (0: from maxn);
//   kind GEMM_KIND_AUTO   gemm_kind(mode, maxn).
// gemm_kind gives each patch's kind by its size: the tensor cores for
// patches of more than 64 DoFs (3xTF32: up to 768), the warp-level MMA
// otherwise.  A patch's arithmetic depends only on its kind, not on nw, maxn
// or the list it is in.  maxn bounds the listed patches' sizes; *status
// (host-mapped) is set to 1 if a tensor-core CTA gave up waiting on one of
// its mbarriers.
enum GemmKind { GEMM_KIND_AUTO = 0, GEMM_KIND_WARP = 1, GEMM_KIND_TC = 2 };
int gemm_kind(int mode, int n);
int gemm_default_warps(int maxn);
void patch_gemm(int mode, int kind, int nw, int nlist, const int* plist, int maxn, int m, const int* poff,
                const int* pdofs, const long long* ioff, const float* inv, const void* tmaps, const void* tmaps_hi,
                const void* tmaps_lo, const float* X, const float* wt, float* Yb, int* status, cudaStream_t s);
// hi[i] = TF32(a[i]) (round to nearest), lo[i] = a[i] - hi[i] (exact): the
// operands of the 3xTF32 tensor-core GEMM
void split_tf32(long long n, const float* a, float* hi, float* lo, cudaStream_t s);

// out[j * m + c] = alpha * sum_{q in slots(j)} Yb[sidx[q] * m + c] + beta * out[j * m + c]
// (slots in increasing order: a fixed summation order)
void pull_scatter(int n, int m, const int* soff, const int* sidx, const float* Yb, float alpha, float beta,
                  float* out, cudaStream_t s);

// E[i * m + c] = sum_j C[i * ldc + j] B[j * m + c] for i, j < nc: the dense
// FP64 coarse inverse applied to a batch (FP64 accumulation).
void coarse_gemm(int nc, int ldc, int m, const double* C, const float* B, float* E, cudaStream_t s);

// ---- FP64 pieces of the batched FGMRES (bkrylov.cu), interleaved [n][m] --
// Y = A X (mode 0) or Y = B - A X (mode 2) with FP64 values
void spmm64(int mode, int nr, int m, const int* rp, const int* ci, const double* av, const double* X, double* Y,
            const double* B, cudaStream_t s);
// doubles of the partial-sum workspace of col_dots at width m
size_t col_partial_doubles(int m);
// out[i][c] (+)= sum_r V_i[r][c] W[r][c] for i < nb (<= 32), basis vectors
// ldv doubles apart; sqrt_out takes the square root (column norms with
// V = W); deterministic (fixed-order two-stage reduction)
void col_dots(int n, int m, int nb, const double* V, long long ldv, const double* W, double* partial, double* out,
              int sqrt_out, int add, cudaStream_t s);
// W[r][c] -= sum_{i < nb} H[i][c] V_i[r][c]
void col_update(int n, int m, int nb, const double* V, long long ldv, const double* H, double* W, cudaStream_t s);
// Vout = W / h[c] per column (0 where h[c] == 0)
void col_scale(int n, int m, const double* W, const double* h, double* Vout, cudaStream_t s);
// per column: Hessenberg column j, Givens rotations, g, |residual estimate|;
// H [m][ldh][ldh], cs / sn [m][ldh], g [m][ldh + 1], hcol [nb][m], hn / resid [m]
void col_givens(int j, int m, int ldh, double* H, const double* hcol, const double* hn, double* cs, double* sn,
                double* g, double* resid, cudaStream_t s);
void col_backsolve(int jend, int m, int ldh, const double* H, const double* g, double* y, cudaStream_t s);
// X[r][c] += sum_{j < jend} y[c][j] Z_j[r][c]; y [m][ldy]
void col_xupdate(int n, int m, int jend, int ldy, const double* Z, long long ldz, const double* y, double* X,
                 cudaStream_t s);
// g[c] = (beta[c], 0, ..., 0), g [m][ldg]
void col_start(int m, int ldg, const double* beta, double* g, cudaStream_t s);
// FP64 [nrhs][n] <-> interleaved [n][m]; FP64 <-> FP32 of an interleaved batch
void pack64(int n, int nrhs, int m, const double* r, double* X, cudaStream_t s);
void unpack64(int n, int nrhs, int m, const double* X, double* z, cudaStream_t s);
void to32(long long nm, const double* x, float* y, cudaStream_t s);
void to64(long long nm, const float* x, double* y, cudaStream_t s);

}  // namespace sbat
