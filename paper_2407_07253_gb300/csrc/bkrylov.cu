// FP64 kernels of the batched FGMRES; see batched.cuh.  Vectors of a batch
// are interleaved DoF-major, X[r * M + c] (DoF r, right-hand side c), so that
// a sparse row or a basis row of all the right-hand sides is one contiguous
// run, and every column is an independent FGMRES (Sec. 4) in lockstep.
#include "batched.cuh"

#include <cmath>

namespace sbat {

namespace {

constexpr int NBMAX = 32;           // basis vectors in one multi-dot (restart + 1 <= 32)
constexpr int DOT_CTAS = 152 * 4;

// Y = A X (MODE 0) or Y = B - A X (MODE 2), FP64; M / 2 lanes per row, one
// double2 of right-hand sides per lane.
template <int MODE>
__global__ void __launch_bounds__(256) k_spmm64(int nr, int m, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const double* __restrict__ av, const double2* __restrict__ X,
                                                double2* __restrict__ Y, const double2* __restrict__ B) {
    const int L = m >> 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long gt = blockIdx.x * (long long)blockDim.x + threadIdx.x; gt < (long long)nr * L; gt += stride) {
        const int row = (int)(gt / L), c2 = (int)(gt - (long long)row * L);
        const int s = __ldg(rp + row), e = __ldg(rp + row + 1);
        double2 acc = make_double2(0.0, 0.0);
        int p = s;
        for (; p + 2 <= e; p += 2) {
            const int c0 = __ldg(ci + p), c1 = __ldg(ci + p + 1);
            const double a0 = __ldg(av + p), a1 = __ldg(av + p + 1);
            const double2 x0 = __ldg(X + (long long)c0 * L + c2), x1 = __ldg(X + (long long)c1 * L + c2);
            acc.x = fma(a0, x0.x, acc.x);
            acc.y = fma(a0, x0.y, acc.y);
            acc.x = fma(a1, x1.x, acc.x);
            acc.y = fma(a1, x1.y, acc.y);
        }
        for (; p < e; ++p) {
            const double a = __ldg(av + p);
            const double2 x = __ldg(X + (long long)__ldg(ci + p) * L + c2);
            acc.x = fma(a, x.x, acc.x);
            acc.y = fma(a, x.y, acc.y);
        }
        if (MODE == 0) Y[gt] = acc;
        else { const double2 b = B[gt]; Y[gt] = make_double2(b.x - acc.x, b.y - acc.y); }
    }
}

// partial[blk][i][c] = sum over the CTA's rows of V_i[r][c] W[r][c], i < nb:
// W is read once, every basis vector once; 256 / M row lanes per CTA.
template <int M>
__global__ void __launch_bounds__(256) k_col_dots(int n, int nb, const double* __restrict__ V, long long ldv,
                                                  const double* __restrict__ W, double* __restrict__ partial) {
    constexpr int RL = 256 / M;
    __shared__ double red[RL][M];
    const int c = threadIdx.x % M, rl = threadIdx.x / M;
    double acc[NBMAX];
#pragma unroll
    for (int i = 0; i < NBMAX; ++i) acc[i] = 0.0;
    for (long long r = (long long)blockIdx.x * RL + rl; r < n; r += (long long)gridDim.x * RL) {
        const double w = W[r * M + c];
#pragma unroll
        for (int i = 0; i < NBMAX; ++i)
            if (i < nb) acc[i] = fma(V[i * ldv + r * M + c], w, acc[i]);
    }
#pragma unroll
    for (int i = 0; i < NBMAX; ++i) {
        if (i < nb) {                       // nb is uniform over the CTA
            red[rl][c] = acc[i];
            __syncthreads();
            if (rl == 0) {
                double s = 0.0;
                for (int q = 0; q < RL; ++q) s += red[q][c];
                partial[((long long)blockIdx.x * NBMAX + i) * M + c] = s;
            }
            __syncthreads();
        }
    }
}

// out[i][c] = sum_blk partial[blk][i][c] in block order (deterministic);
// sqrt_out: out = sqrt(out) (column norms); add: out += that sum
__global__ void k_col_reduce(int nblk, int nb, int m, const double* __restrict__ partial, double* __restrict__ out,
                             int sqrt_out, int add) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * m) return;
    const int i = t / m, c = t - i * m;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[((long long)b * NBMAX + i) * m + c];
    if (sqrt_out) s = sqrt(s);
    out[t] = add ? out[t] + s : s;
}

// W[r][c] -= sum_{i < nb} H[i][c] V_i[r][c]
__global__ void k_col_update(long long nm, int m, int nb, const double* __restrict__ V, long long ldv,
                             const double* __restrict__ H, double* __restrict__ W) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % m);
        double s = W[t];
        for (int i = 0; i < nb; ++i) s = fma(-H[i * m + c], V[i * ldv + t], s);
        W[t] = s;
    }
}

// Vout[r][c] = W[r][c] / h[c] (0 where h[c] == 0: a column already exact)
__global__ void k_col_scale(long long nm, int m, const double* __restrict__ W, const double* __restrict__ h,
                            double* __restrict__ Vout) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x) {
        const double d = h[t % m];
        Vout[t] = d > 0.0 ? W[t] / d : 0.0;
    }
}

// one column c per thread: append (hcol[.][c], hn[c]) as column j of the
// column's Hessenberg matrix, apply the previous rotations, form the next,
// update g and the residual estimate (the single-RHS fgmres_givens per column)
__global__ void k_col_givens(int j, int m, int ldh, double* __restrict__ H, const double* __restrict__ hcol,
                             const double* __restrict__ hn, double* __restrict__ cs, double* __restrict__ sn,
                             double* __restrict__ g, double* __restrict__ resid) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double* Hc = H + (long long)c * ldh * ldh;
    double* csc = cs + (long long)c * ldh;
    double* snc = sn + (long long)c * ldh;
    double* gc = g + (long long)c * (ldh + 1);
    for (int i = 0; i <= j; ++i) Hc[i * ldh + j] = hcol[i * m + c];
    Hc[(j + 1) * ldh + j] = hn[c];
    for (int i = 0; i < j; ++i) {
        const double a = Hc[i * ldh + j], b = Hc[(i + 1) * ldh + j];
        Hc[i * ldh + j] = csc[i] * a + snc[i] * b;
        Hc[(i + 1) * ldh + j] = -snc[i] * a + csc[i] * b;
    }
    const double a = Hc[j * ldh + j], b = Hc[(j + 1) * ldh + j];
    const double den = hypot(a, b);
    double cc = 1.0, ss = 0.0;
    if (den > 0.0) { cc = a / den; ss = b / den; }
    csc[j] = cc;
    snc[j] = ss;
    Hc[j * ldh + j] = den > 0.0 ? den : a;
    Hc[(j + 1) * ldh + j] = 0.0;
    gc[j + 1] = -ss * gc[j];
    gc[j] = cc * gc[j];
    resid[c] = fabs(gc[j + 1]);
}

// y = H^-1 g per column (upper triangular, jend columns); a zero pivot (a
// column whose Krylov space was exhausted earlier) contributes y = 0
__global__ void k_col_backsolve(int jend, int m, int ldh, const double* __restrict__ H, const double* __restrict__ g,
                                double* __restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const double* Hc = H + (long long)c * ldh * ldh;
    const double* gc = g + (long long)c * (ldh + 1);
    double* yc = y + (long long)c * (ldh + 1);
    for (int i = jend - 1; i >= 0; --i) {
        double s = gc[i];
        for (int l = i + 1; l < jend; ++l) s -= Hc[i * ldh + l] * yc[l];
        yc[i] = Hc[i * ldh + i] != 0.0 ? s / Hc[i * ldh + i] : 0.0;
    }
}

// X[r][c] += sum_{j < jend} y[c][j] Z_j[r][c]
__global__ void k_col_xupdate(long long nm, int m, int jend, int ldy, const double* __restrict__ Z, long long ldz,
                              const double* __restrict__ y, double* __restrict__ X) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % m);
        double s = X[t];
        for (int j = 0; j < jend; ++j) s = fma(y[(long long)c * ldy + j], Z[j * ldz + t], s);
        X[t] = s;
    }
}

// g[c][0] = beta[c], the rest 0; V0[r][c] = R[r][c] / beta[c]
__global__ void k_col_start(int m, int ldg, const double* __restrict__ beta, double* __restrict__ g) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * ldg) return;
    const int c = t / ldg, i = t - c * ldg;
    g[t] = i == 0 ? beta[c] : 0.0;
}

// FP64 [nrhs][n] <-> FP64 interleaved [n][m] (zero columns nrhs .. m - 1)
__global__ void k_pack64(int n, int nrhs, int m, const double* __restrict__ r, double* __restrict__ X) {
    const long long total = (long long)n * m;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(t / m), c = (int)(t - (long long)j * m);
        X[t] = c < nrhs ? r[(long long)c * n + j] : 0.0;
    }
}
__global__ void k_unpack64(int n, int nrhs, int m, const double* __restrict__ X, double* __restrict__ z) {
    const long long total = (long long)n * nrhs;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t / n), j = (int)(t - (long long)c * n);
        z[t] = X[(long long)j * m + c];
    }
}
// FP64 interleaved <-> FP32 interleaved (same layout)
__global__ void k_to32(long long nm, const double* __restrict__ x, float* __restrict__ y) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x)
        y[t] = (float)x[t];
}
__global__ void k_to64(long long nm, const float* __restrict__ x, double* __restrict__ y) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nm; t += (long long)gridDim.x * blockDim.x)
        y[t] = (double)x[t];
}

inline int grid_of(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

template <int M>
void col_dots_m(int n, int nb, const double* V, long long ldv, const double* W, double* partial, double* out,
                int sqrt_out, int add, cudaStream_t s) {
    k_col_dots<M><<<DOT_CTAS, 256, 0, s>>>(n, nb, V, ldv, W, partial);
    k_col_reduce<<<(nb * M + 255) / 256, 256, 0, s>>>(DOT_CTAS, nb, M, partial, out, sqrt_out, add);
}

}  // namespace

size_t col_partial_doubles(int m) { return (size_t)DOT_CTAS * NBMAX * m; }

void spmm64(int mode, int nr, int m, const int* rp, const int* ci, const double* av, const double* X, double* Y,
            const double* B, cudaStream_t s) {
    const int grid = grid_of((long long)nr * (m / 2));
    const double2* X2 = reinterpret_cast<const double2*>(X);
    double2* Y2 = reinterpret_cast<double2*>(Y);
    const double2* B2 = reinterpret_cast<const double2*>(B);
    if (mode == 0) k_spmm64<0><<<grid, 256, 0, s>>>(nr, m, rp, ci, av, X2, Y2, B2);
    else k_spmm64<2><<<grid, 256, 0, s>>>(nr, m, rp, ci, av, X2, Y2, B2);
}

void col_dots(int n, int m, int nb, const double* V, long long ldv, const double* W, double* partial, double* out,
              int sqrt_out, int add, cudaStream_t s) {
    switch (m) {
        case 8: col_dots_m<8>(n, nb, V, ldv, W, partial, out, sqrt_out, add, s); break;
        case 16: col_dots_m<16>(n, nb, V, ldv, W, partial, out, sqrt_out, add, s); break;
        case 32: col_dots_m<32>(n, nb, V, ldv, W, partial, out, sqrt_out, add, s); break;
        default: col_dots_m<64>(n, nb, V, ldv, W, partial, out, sqrt_out, add, s); break;
    }
}

void col_update(int n, int m, int nb, const double* V, long long ldv, const double* H, double* W, cudaStream_t s) {
    const long long nm = (long long)n * m;
    k_col_update<<<grid_of(nm), 256, 0, s>>>(nm, m, nb, V, ldv, H, W);
}

void col_scale(int n, int m, const double* W, const double* h, double* Vout, cudaStream_t s) {
    const long long nm = (long long)n * m;
    k_col_scale<<<grid_of(nm), 256, 0, s>>>(nm, m, W, h, Vout);
}

void col_givens(int j, int m, int ldh, double* H, const double* hcol, const double* hn, double* cs, double* sn,
                double* g, double* resid, cudaStream_t s) {
    k_col_givens<<<(m + 63) / 64, 64, 0, s>>>(j, m, ldh, H, hcol, hn, cs, sn, g, resid);
}

void col_backsolve(int jend, int m, int ldh, const double* H, const double* g, double* y, cudaStream_t s) {
    k_col_backsolve<<<(m + 63) / 64, 64, 0, s>>>(jend, m, ldh, H, g, y);
}

void col_xupdate(int n, int m, int jend, int ldy, const double* Z, long long ldz, const double* y, double* X,
                 cudaStream_t s) {
    const long long nm = (long long)n * m;
    k_col_xupdate<<<grid_of(nm), 256, 0, s>>>(nm, m, jend, ldy, Z, ldz, y, X);
}

void col_start(int m, int ldg, const double* beta, double* g, cudaStream_t s) {
    k_col_start<<<(m * ldg + 255) / 256, 256, 0, s>>>(m, ldg, beta, g);
}

void pack64(int n, int nrhs, int m, const double* r, double* X, cudaStream_t s) {
    k_pack64<<<grid_of((long long)n * m), 256, 0, s>>>(n, nrhs, m, r, X);
}

void unpack64(int n, int nrhs, int m, const double* X, double* z, cudaStream_t s) {
    k_unpack64<<<grid_of((long long)n * nrhs), 256, 0, s>>>(n, nrhs, m, X, z);
}

void to32(long long nm, const double* x, float* y, cudaStream_t s) { k_to32<<<grid_of(nm), 256, 0, s>>>(nm, x, y); }
void to64(long long nm, const float* x, double* y, cudaStream_t s) { k_to64<<<grid_of(nm), 256, 0, s>>>(nm, x, y); }

}  // namespace sbat
