// Device assembly of the Stokes operator and matrix-free load vector; see
// assembly.cuh.
#include "assembly.cuh"

#include <algorithm>

#include <climits>

namespace sasm {

namespace {

constexpr int WARPS = 4;               // warps per block, one node per warp
constexpr unsigned FULL = 0xffffffffu;

// one thread per cell: the factors described with CG_STRIDE
__global__ void k_cell_geometry(AsmMesh m, double* cg) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m.nc) return;
    const int d = m.d;
    const int* v = m.C + (long long)e * (d + 1);
    double J[9];
    for (int c = 0; c < d; ++c)
        for (int a = 0; a < d; ++a) J[c * d + a] = m.X[(long long)v[a + 1] * d + c] - m.X[(long long)v[0] * d + c];
    double adj[9], det;
    if (d == 2) {
        det = J[0] * J[3] - J[1] * J[2];
        adj[0] = J[3];  adj[1] = -J[1];
        adj[2] = -J[2]; adj[3] = J[0];
    } else {
        const double a = J[0], b = J[1], c = J[2], dd = J[3], e2 = J[4], f = J[5], gg = J[6], h = J[7], i = J[8];
        const double A = e2 * i - f * h, B = -(dd * i - f * gg), Cc = dd * h - e2 * gg;
        det = a * A + b * B + c * Cc;
        const double t[9] = {A, -(b * i - c * h), b * f - c * e2, B, a * i - c * gg, -(a * f - c * dd),
                             Cc, -(a * h - b * gg), a * e2 - b * dd};
        for (int k = 0; k < 9; ++k) adj[k] = t[k];
    }
    const double rdet = 1.0 / det, adet = fabs(det);
    double Ji[9];
    for (int k = 0; k < d * d; ++k) Ji[k] = adj[k] * rdet;   // Jinv[a][c] = d xi_a / d x_c
    double* o = cg + (long long)e * CG_STRIDE;
    const double wgt = adet * (m.nu ? m.nu[e] : 1.0);
    o[0] = adet;
    for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
            double s = 0;
            for (int c = 0; c < d; ++c) s += Ji[a * d + c] * Ji[b * d + c];
            o[1 + a * d + b] = wgt * s;
        }
    for (int a = 0; a < d; ++a)
        for (int c = 0; c < d; ++c) o[1 + d * d + a * d + c] = -adet * Ji[a * d + c];
}

// Warp-cooperative insertion of this lane's candidate into the list of
// distinct values (first-appearance order).  *where receives the candidate's
// position in the list (-1 if !valid).  Returns false on overflow.
__device__ bool warp_insert(int* list, int* cnt, int cap, int cand, bool valid, int* where) {
    const int lane = threadIdx.x & 31;
    const int n0 = *cnt;
    bool keep = valid;
    int found = -1;
    if (keep)
        for (int t = 0; t < n0; ++t)
            if (list[t] == cand) { keep = false; found = t; break; }
    const unsigned same = __match_any_sync(FULL, keep ? cand : INT_MIN + lane);
    const int leader = __ffs(same) - 1;
    keep = keep && (lane == leader);
    const unsigned km = __ballot_sync(FULL, keep);
    const int pos = n0 + __popc(km & ((1u << lane) - 1u));
    const bool ok = n0 + __popc(km) <= cap;
    if (keep && ok) list[pos] = cand;
    // a new value's position is its group leader's
    const int lpos = __shfl_sync(FULL, pos, leader);
    *where = !valid ? -1 : (found >= 0 ? found : lpos);
    __syncwarp();
    if (lane == 0) *cnt = ok ? n0 + __popc(km) : cap + 1;
    __syncwarp();
    return ok;
}

// neighbours of node `node` whose incident cells are adj[off[node] .. ):
// free velocity nodes into lv, pressure nodes into lq (if lq != nullptr).
// With pv (pq) != nullptr, pv[c * nb + b] receives the list position of
// velocity node b of incident cell c (-1: not free), pq likewise for the
// pressure nodes; the caller passes them when every incident (cell, node)
// pair fits in MAX_POS.
__device__ bool neighbours(const AsmMesh& m, const int* off, const int* adj, int per_cell, int node, int* lv,
                           int* cv, int* lq, int* cq, short* pv = nullptr, short* pq = nullptr) {
    const int lane = threadIdx.x & 31;
    const int c0 = off[node], ncell = off[node + 1] - c0;
    if (lane == 0) { *cv = 0; if (lq) *cq = 0; }
    __syncwarp();
    const int tv = ncell * m.nb;
    for (int base = 0; base < tv; base += 32) {
        const int t = base + lane;
        int cand = 0;
        bool valid = false;
        if (t < tv) {
            const int e = adj[c0 + t / m.nb] / per_cell;
            cand = m.vcell[(long long)e * m.nb + t % m.nb];
            valid = m.vfree[cand] >= 0;
        }
        int where;
        if (!warp_insert(lv, cv, m.cap_v, cand, valid, &where)) return false;
        if (pv && t < tv) pv[t] = (short)where;
    }
    if (lq) {
        const int tq = ncell * m.nq;
        for (int base = 0; base < tq; base += 32) {
            const int t = base + lane;
            int cand = 0;
            bool valid = false;
            if (t < tq) {
                const int e = adj[c0 + t / m.nq] / per_cell;
                cand = m.qcell[(long long)e * m.nq + t % m.nq];
                valid = true;
            }
            int where;
            if (!warp_insert(lq, cq, m.cap_q, cand, valid, &where)) return false;
            if (pq && t < tq) pq[t] = (short)where;
        }
    }
    return true;
}

__device__ int find(const int* list, int n, int x) {
    for (int t = 0; t < n; ++t)
        if (list[t] == x) return t;
    return -1;
}

// incident (cell, node) pairs of one node whose list positions are kept
// (rows with more use a search of the list)
constexpr int MAX_POS = 256;

// One warp's lists in dynamic shared memory: the two counts, the velocity
// and pressure neighbour lists (cap_v, cap_q entries) and the position maps
// (min(cap, MAX_POS) entries each), 16-byte aligned per warp.
struct WarpLists {
    int* lv;
    int* lq;
    short* pv;
    short* pq;
    int* cv;
    int* cq;
    int npv, npq;                      // entries of pv, pq
};
__host__ __device__ inline size_t warp_list_bytes(int cap_v, int cap_q) {
    const int npv = cap_v < MAX_POS ? cap_v : MAX_POS, npq = cap_q < MAX_POS ? cap_q : MAX_POS;
    const size_t b = 8 + 4 * (size_t)(cap_v + cap_q) + 2 * (size_t)(npv + npq);
    return (b + 15) & ~(size_t)15;
}
__device__ WarpLists warp_lists(const AsmMesh& m, int w) {
    extern __shared__ int4 asm_smem[];
    char* p = reinterpret_cast<char*>(asm_smem) + (size_t)w * warp_list_bytes(m.cap_v, m.cap_q);
    WarpLists L;
    L.npv = m.cap_v < MAX_POS ? m.cap_v : MAX_POS;
    L.npq = m.cap_q < MAX_POS ? m.cap_q : MAX_POS;
    L.cv = reinterpret_cast<int*>(p);
    L.cq = L.cv + 1;
    L.lv = L.cv + 2;
    L.lq = L.lv + m.cap_v;
    L.pv = reinterpret_cast<short*>(L.lq + m.cap_q);
    L.pq = L.pv + L.npv;
    return L;
}

__global__ void __launch_bounds__(WARPS * 32) k_row_lengths(AsmMesh m, int* len, int* status) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * WARPS + w;
    const WarpLists L = warp_lists(m, w);
    if (item < m.nVf) {
        const int node = m.vrow[item];
        if (!neighbours(m, m.voff, m.vadj, m.nb, node, L.lv, L.cv, L.lq, L.cq)) {
            if (lane == 0) atomicExch(status, 1);
            return;
        }
        if (lane == 0)
            for (int c = 0; c < m.d; ++c) len[c * m.nVf + item] = *L.cv + *L.cq;
    } else if (item < m.nVf + m.nQ) {
        const int q = item - m.nVf;
        if (!neighbours(m, m.qoff, m.qadj, m.nq, q, L.lv, L.cv, nullptr, nullptr)) {
            if (lane == 0) atomicExch(status, 1);
            return;
        }
        if (lane == 0) len[m.d * m.nVf + q] = m.d * *L.cv;
    }
}

// Values accumulate directly in the output row segments: a warp owns its
// rows, lanes of one cell touch distinct positions, and __syncwarp orders the
// cells, so the sums are deterministic without atomics.
__global__ void __launch_bounds__(WARPS * 32) k_fill(AsmMesh m, const int* rp, int* ci, double* val, int* status) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * WARPS + w;
    const WarpLists L = warp_lists(m, w);
    const int d = m.d, nb = m.nb, nq = m.nq;
    if (item < m.nVf) {
        const int node = m.vrow[item];
        const int ncell = m.voff[node + 1] - m.voff[node];
        const bool map = ncell * nb <= L.npv && ncell * nq <= L.npq;
        if (!neighbours(m, m.voff, m.vadj, nb, node, L.lv, L.cv, L.lq, L.cq, map ? L.pv : nullptr,
                        map ? L.pq : nullptr)) {
            if (lane == 0) atomicExch(status, 1);
            return;
        }
        const int cv = *L.cv, cq = *L.cq;
        const int len = cv + cq;
        for (int c = 0; c < d; ++c) {
            const long long r0 = rp[c * m.nVf + item];
            for (int t = lane; t < len; t += 32) {
                val[r0 + t] = 0.0;
                ci[r0 + t] = t < cv ? c * m.nVf + m.vfree[L.lv[t]] : d * m.nVf + L.lq[t - cv];
            }
        }
        __syncwarp();
        const long long r00 = rp[item];
        for (int x = m.voff[node]; x < m.voff[node + 1]; ++x) {
            const int e = m.vadj[x] / nb, la = m.vadj[x] % nb, xl = x - m.voff[node];
            const double* G = m.cg + (long long)e * CG_STRIDE + 1;      // weighted stiffness factors
            const double* D = G + d * d;                                // divergence factors
            for (int b = lane; b < nb; b += 32) {
                const int j = m.vcell[(long long)e * nb + b];
                if (m.vfree[j] < 0) continue;
                double s = 0;
                for (int a = 0; a < d; ++a)
                    for (int bb = 0; bb < d; ++bb) s += G[a * d + bb] * m.S[(((long long)a * d + bb) * nb + la) * nb + b];
                val[r00 + (map ? L.pv[xl * nb + b] : find(L.lv, cv, j))] += s;
            }
            for (int p = lane; p < nq; p += 32) {
                const int q = m.qcell[(long long)e * nq + p];
                const int pos = cv + (map ? L.pq[xl * nq + p] : find(L.lq, cq, q));
                for (int c = 0; c < d; ++c) {
                    double s = 0;
                    for (int a = 0; a < d; ++a) s += D[a * d + c] * m.Cq[((long long)a * nq + p) * nb + la];
                    val[rp[c * m.nVf + item] + pos] += s;
                }
            }
            __syncwarp();
        }
        // the velocity block is the same for every component
        for (int c = 1; c < d; ++c) {
            const long long r0 = rp[c * m.nVf + item];
            for (int t = lane; t < cv; t += 32) val[r0 + t] = val[r00 + t];
        }
    } else if (item < m.nVf + m.nQ) {
        const int q = item - m.nVf;
        const int ncell = m.qoff[q + 1] - m.qoff[q];
        const bool map = ncell * nb <= L.npv;
        if (!neighbours(m, m.qoff, m.qadj, nq, q, L.lv, L.cv, nullptr, nullptr, map ? L.pv : nullptr)) {
            if (lane == 0) atomicExch(status, 1);
            return;
        }
        const int cv = *L.cv;
        const long long r0 = rp[d * m.nVf + q];
        for (int c = 0; c < d; ++c)
            for (int t = lane; t < cv; t += 32) {
                ci[r0 + (long long)c * cv + t] = c * m.nVf + m.vfree[L.lv[t]];
                val[r0 + (long long)c * cv + t] = 0.0;
            }
        __syncwarp();
        for (int x = m.qoff[q]; x < m.qoff[q + 1]; ++x) {
            const int e = m.qadj[x] / nq, lp = m.qadj[x] % nq, xl = x - m.qoff[q];
            const double* D = m.cg + (long long)e * CG_STRIDE + 1 + d * d;
            for (int b = lane; b < nb; b += 32) {
                const int j = m.vcell[(long long)e * nb + b];
                if (m.vfree[j] < 0) continue;
                const int pos = map ? L.pv[xl * nb + b] : find(L.lv, cv, j);
                for (int c = 0; c < d; ++c) {
                    double s = 0;
                    for (int a = 0; a < d; ++a) s += D[a * d + c] * m.Cq[((long long)a * nq + lp) * nb + b];
                    val[r0 + (long long)c * cv + pos] += s;
                }
            }
            __syncwarp();
        }
    }
}

// exclusive scan, 1024 elements per block
__global__ void __launch_bounds__(1024) k_scan_block(const int* in, int n, int* out, int* bsum) {
    __shared__ int ws[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = i < n ? in[i] : 0;
    int v = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = ws[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const int incl = v + (w > 0 ? ws[w - 1] : 0);
    if (i < n) out[i] = incl - x;
    if (threadIdx.x == 1023) bsum[blockIdx.x] = incl;
}

__global__ void k_scan_sums(int* bsum, int nb) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int run = 0;
    for (int b = 0; b < nb; ++b) {
        const int t = bsum[b];
        bsum[b] = run;
        run += t;
    }
    bsum[nb] = run;
}

__global__ void k_scan_add(int* out, int n, const int* bsum, int nblk) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / 1024];
    if (i == 0) out[n] = bsum[nblk];
}

// one thread per row: b = (M f)/nu on velocity rows minus K[r, D] g
__global__ void k_load(AsmMesh m, const double* f, const double* gD, double inv_nu, double* b) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int d = m.d, nb = m.nb, nq = m.nq;
    if (r < d * m.nVf) {
        const int c = r / m.nVf, fi = r - c * m.nVf;
        const int node = m.vrow[fi];
        double F = 0, lift = 0;
        for (int x = m.voff[node]; x < m.voff[node + 1]; ++x) {
            const int e = m.vadj[x] / nb, la = m.vadj[x] % nb;
            const double* cge = m.cg + (long long)e * CG_STRIDE;
            double Fe = 0;
            for (int bb = 0; bb < nb; ++bb) {
                const int j = m.vcell[(long long)e * nb + bb];
                Fe += m.M[(long long)la * nb + bb] * f[(long long)c * m.nV + j];
            }
            F += cge[0] * Fe;
            if (gD) {
                const double* G = cge + 1;
                for (int bb = 0; bb < nb; ++bb) {
                    const int j = m.vcell[(long long)e * nb + bb];
                    if (m.vfree[j] >= 0) continue;
                    double s = 0;
                    for (int a = 0; a < d; ++a)
                        for (int a2 = 0; a2 < d; ++a2) s += G[a * d + a2] * m.S[(((long long)a * d + a2) * nb + la) * nb + bb];
                    lift += s * gD[(long long)c * m.nV + j];
                }
            }
        }
        b[r] = F * inv_nu - lift;
    } else if (r < d * m.nVf + m.nQ) {
        const int q = r - d * m.nVf;
        double lift = 0;
        if (gD)
            for (int x = m.qoff[q]; x < m.qoff[q + 1]; ++x) {
                const int e = m.qadj[x] / nq, lp = m.qadj[x] % nq;
                const double* D = m.cg + (long long)e * CG_STRIDE + 1 + d * d;
                for (int bb = 0; bb < nb; ++bb) {
                    const int j = m.vcell[(long long)e * nb + bb];
                    if (m.vfree[j] >= 0) continue;
                    for (int c = 0; c < d; ++c) {
                        double s = 0;
                        for (int a = 0; a < d; ++a) s += D[a * d + c] * m.Cq[((long long)a * nq + lp) * nb + bb];
                        lift += s * gD[(long long)c * m.nV + j];
                    }
                }
            }
        b[r] = -lift;
    }
}

// dL/dnu_e = -sum_q lambda_q,e^T A_e u_q,e summed over the velocity
// components and the nq (u, lambda) pairs of a batch, A_e the cell's
// unit-viscosity scalar stiffness (the operator's A_e(nu_e) = nu_e A_e, so the
// stored factors are divided by nu_e).  One warp per cell: up to GQ_MAX
// columns' velocities are staged in shared memory at a time, lane i takes
// element row i, forms A_e[i][j] = sum_ab G_ab S_ab[i][j] on the fly once per
// pass (the same for every component and column) and pairs it with
// sum_q,c lambda_q,c[i] u_q,c[j]; a warp sum ends it.
constexpr int GQ_MAX = 4;

__global__ void __launch_bounds__(256) k_grad_nu(AsmMesh m, const double* __restrict__ u,
                                                 const double* __restrict__ lam, int nq, long long ld, int gq,
                                                 double* __restrict__ grad) {
    extern __shared__ double us_all[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, d = m.d, nb = m.nb, dnb = d * nb;
    double* us = us_all + (size_t)w * gq * dnb;
    for (int e = blockIdx.x * 8 + w; e < m.nc; e += gridDim.x * 8) {
        const int* vc = m.vcell + (long long)e * nb;
        const double* G = m.cg + (long long)e * CG_STRIDE + 1;
        double acc = 0;
        for (int q0 = 0; q0 < nq; q0 += gq) {
            const int nqc = min(gq, nq - q0);
            for (int t = lane; t < nqc * dnb; t += 32) {
                const int qq = t / dnb, r = t - qq * dnb, c = r / nb, j = r - c * nb;
                us[t] = u[(q0 + qq) * ld + (long long)c * m.nV + vc[j]];
            }
            __syncwarp();
            for (int i = lane; i < nb; i += 32) {
                const int node = vc[i];
                double li[GQ_MAX][3];
#pragma unroll
                for (int qq = 0; qq < GQ_MAX; ++qq)
                    for (int c = 0; c < 3; ++c)
                        li[qq][c] = (qq < nqc && c < d) ? lam[(q0 + qq) * ld + (long long)c * m.nV + node] : 0.0;
                for (int j = 0; j < nb; ++j) {
                    double aij = 0;
                    for (int a = 0; a < d; ++a)
                        for (int a2 = 0; a2 < d; ++a2) aij += G[a * d + a2] * m.S[(((long long)a * d + a2) * nb + i) * nb + j];
                    double sj = 0;
#pragma unroll
                    for (int qq = 0; qq < GQ_MAX; ++qq)
                        if (qq < nqc)
                            for (int c = 0; c < d; ++c) sj += li[qq][c] * us[(qq * d + c) * nb + j];
                    acc += aij * sj;
                }
            }
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) grad[e] = -acc / (m.nu ? m.nu[e] : 1.0);
        __syncwarp();
    }
}

// out[c][i] = scale (M lambda_c)[i] on every velocity node, pulled over the
// node's cells in adjacency order (deterministic)
__global__ void k_mass_all(AsmMesh m, const double* __restrict__ lam, double scale, double* __restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)m.d * m.nV) return;
    const int c = (int)(t / m.nV), node = (int)(t - (long long)c * m.nV), nb = m.nb;
    double F = 0;
    for (int x = m.voff[node]; x < m.voff[node + 1]; ++x) {
        const int e = m.vadj[x] / nb, la = m.vadj[x] % nb;
        double Fe = 0;
        for (int bb = 0; bb < nb; ++bb)
            Fe += m.M[(long long)la * nb + bb] * lam[(long long)c * m.nV + m.vcell[(long long)e * nb + bb]];
        F += m.cg[(long long)e * CG_STRIDE] * Fe;
    }
    out[t] = scale * F;
}

// ---- device interpolation
__global__ void k_interp_rows(InterpGeom g, InterpSpace F, InterpSpace C, int nrows, const int* __restrict__ rows,
                              int* __restrict__ cnt, int* __restrict__ col, double* __restrict__ val) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= nrows) return;
    const int node = rows ? rows[row] : row;
    const int first = F.adj[F.off[node]];
    const int e = first / F.nb, l = first - e * F.nb;
    const int nbc = C.nb, d = g.d;
    double v[INTERP_MAX_NB];
    int cc = e;
    if (!g.nested) {
        for (int b = 0; b < nbc; ++b) v[b] = g.tab[l * nbc + b];
    } else {
        cc = g.parent[e];
        // the fine node: x = x_0 + sum_a (alpha_a / k_f) (x_a - x_0) on its owner cell
        double x[3] = {0, 0, 0};
        const int* fv = g.Cf + (long long)e * (d + 1);
        for (int c = 0; c < d; ++c) {
            const double x0 = g.Xf[(long long)fv[0] * d + c];
            double s = x0;
            for (int a = 1; a <= d; ++a)
                s += (double)g.alpha_f[l * 4 + a] / g.kf * (g.Xf[(long long)fv[a] * d + c] - x0);
            x[c] = s;
        }
        // its reference coordinates in the coarse cell: xi = J^-1 (x - x_0)
        const int* cv = g.Cc + (long long)cc * (d + 1);
        double J[9], xi[3] = {0, 0, 0}, rhs[3];
        for (int c = 0; c < d; ++c) {
            const double x0 = g.Xc[(long long)cv[0] * d + c];
            rhs[c] = x[c] - x0;
            for (int a = 0; a < d; ++a) J[c * d + a] = g.Xc[(long long)cv[a + 1] * d + c] - x0;
        }
        if (d == 2) {
            const double det = J[0] * J[3] - J[1] * J[2];
            xi[0] = (J[3] * rhs[0] - J[1] * rhs[1]) / det;
            xi[1] = (-J[2] * rhs[0] + J[0] * rhs[1]) / det;
        } else {
            const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
            const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
            const double i00 = c00 / det, i01 = (J[2] * J[7] - J[1] * J[8]) / det, i02 = (J[1] * J[5] - J[2] * J[4]) / det;
            const double i10 = c01 / det, i11 = (J[0] * J[8] - J[2] * J[6]) / det, i12 = (J[2] * J[3] - J[0] * J[5]) / det;
            const double i20 = c02 / det, i21 = (J[1] * J[6] - J[0] * J[7]) / det, i22 = (J[0] * J[4] - J[1] * J[3]) / det;
            xi[0] = i00 * rhs[0] + i01 * rhs[1] + i02 * rhs[2];
            xi[1] = i10 * rhs[0] + i11 * rhs[1] + i12 * rhs[2];
            xi[2] = i20 * rhs[0] + i21 * rhs[1] + i22 * rhs[2];
        }
        for (int b = 0; b < nbc; ++b) v[b] = 0.0;
        for (int m = 0; m < g.nm; ++m) {
            double mv = 1.0;
            for (int a = 0; a < d; ++a)
                for (int t = 0; t < g.mono[m * 3 + a]; ++t) mv *= xi[a];
            for (int b = 0; b < nbc; ++b) v[b] += g.coef[b * g.nm + m] * mv;
        }
    }
    // entries on free coarse nodes, sorted by column (insertion sort)
    int* cr = col + (long long)row * nbc;
    double* vr = val + (long long)row * nbc;
    int m = 0;
    for (int b = 0; b < nbc; ++b) {
        if (!(fabs(v[b]) > 1e-14)) continue;
        const int cn = C.cell[(long long)cc * nbc + b];
        const int cf = C.free ? C.free[cn] : cn;
        if (cf < 0) continue;
        int t = m++;
        while (t > 0 && cr[t - 1] > cf) { cr[t] = cr[t - 1]; vr[t] = vr[t - 1]; --t; }
        cr[t] = cf;
        vr[t] = v[b];
    }
    cnt[row] = m;
}

__global__ void k_interp_lengths(int d, int nVf, int nQf, const int* __restrict__ cntV, const int* __restrict__ cntQ,
                                 int* __restrict__ len) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int nr = d * nVf + nQf;
    if (r >= nr) return;
    len[r] = r < d * nVf ? cntV[r % nVf] : cntQ[r - d * nVf];
}

__global__ void k_interp_fill(int d, int nVf, int nQf, int nVf_c, int sV, int sQ, const int* __restrict__ cntV,
                              const int* __restrict__ colV, const double* __restrict__ valV,
                              const int* __restrict__ cntQ, const int* __restrict__ colQ,
                              const double* __restrict__ valQ, const int* __restrict__ rp, int* __restrict__ ci,
                              double* __restrict__ v) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int nr = d * nVf + nQf;
    if (r >= nr) return;
    int o = rp[r];
    if (r < d * nVf) {
        const int c = r / nVf, f = r - c * nVf;
        for (int t = 0; t < cntV[f]; ++t, ++o) {
            ci[o] = c * nVf_c + colV[(long long)f * sV + t];
            v[o] = valV[(long long)f * sV + t];
        }
    } else {
        const int q = r - d * nVf;
        for (int t = 0; t < cntQ[q]; ++t, ++o) {
            ci[o] = d * nVf_c + colQ[(long long)q * sQ + t];
            v[o] = valQ[(long long)q * sQ + t];
        }
    }
}

__global__ void k_transpose_count(int nr, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ cnt) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    for (int p = rp[r]; p < rp[r + 1]; ++p) atomicAdd(&cnt[ci[p]], 1);
}

__global__ void k_transpose_fill(int nr, const int* __restrict__ rp, const int* __restrict__ ci,
                                 const double* __restrict__ v, const int* __restrict__ rrp, int* __restrict__ cur,
                                 int* __restrict__ rci, double* __restrict__ rv) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    for (int p = rp[r]; p < rp[r + 1]; ++p) {
        const int c = ci[p];
        const int o = rrp[c] + atomicAdd(&cur[c], 1);
        rci[o] = r;
        rv[o] = v[p];
    }
}

// each row's entries sorted by column (insertion sort; rows are short)
__global__ void k_sort_rows(int nr, const int* __restrict__ rp, int* __restrict__ ci, double* __restrict__ v) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const int s = rp[r], e = rp[r + 1];
    for (int p = s + 1; p < e; ++p) {
        const int c = ci[p];
        const double x = v[p];
        int q = p;
        while (q > s && ci[q - 1] > c) { ci[q] = ci[q - 1]; v[q] = v[q - 1]; --q; }
        ci[q] = c;
        v[q] = x;
    }
}

__global__ void k_to_float(long long n, const double* __restrict__ x, float* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)x[i];
}

}  // namespace

void interp_rows(const InterpGeom& g, const InterpSpace& fine, const InterpSpace& coarse, int nrows, const int* rows,
                 int* cnt, int* col, double* val, cudaStream_t s) {
    if (nrows <= 0) return;
    k_interp_rows<<<(nrows + 127) / 128, 128, 0, s>>>(g, fine, coarse, nrows, rows, cnt, col, val);
}
void interp_lengths(int d, int nVf, int nQf, const int* cntV, const int* cntQ, int* len, cudaStream_t s) {
    const int nr = d * nVf + nQf;
    if (nr > 0) k_interp_lengths<<<(nr + 255) / 256, 256, 0, s>>>(d, nVf, nQf, cntV, cntQ, len);
}
void interp_fill(int d, int nVf, int nQf, int nVf_c, int sV, int sQ, const int* cntV, const int* colV,
                 const double* valV, const int* cntQ, const int* colQ, const double* valQ, const int* rp, int* ci,
                 double* v, cudaStream_t s) {
    const int nr = d * nVf + nQf;
    if (nr > 0)
        k_interp_fill<<<(nr + 255) / 256, 256, 0, s>>>(d, nVf, nQf, nVf_c, sV, sQ, cntV, colV, valV, cntQ, colQ, valQ,
                                                         rp, ci, v);
}
void transpose_count(int nr, const int* rp, const int* ci, int ncol, int* cnt, cudaStream_t s) {
    cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)ncol, s);
    if (nr > 0) k_transpose_count<<<(nr + 255) / 256, 256, 0, s>>>(nr, rp, ci, cnt);
}
void transpose_fill(int nr, const int* rp, const int* ci, const double* v, int ncol, const int* rrp, int* cur,
                    int* rci, double* rv, cudaStream_t s) {
    cudaMemsetAsync(cur, 0, sizeof(int) * (size_t)ncol, s);
    if (nr > 0) k_transpose_fill<<<(nr + 255) / 256, 256, 0, s>>>(nr, rp, ci, v, rrp, cur, rci, rv);
}
void sort_rows(int nr, const int* rp, int* ci, double* v, cudaStream_t s) {
    if (nr > 0) k_sort_rows<<<(nr + 255) / 256, 256, 0, s>>>(nr, rp, ci, v);
}
void to_float(long long n, const double* x, float* y, cudaStream_t s) {
    if (n > 0) k_to_float<<<(int)std::min<long long>((n + 255) / 256, 152LL * 16), 256, 0, s>>>(n, x, y);
}

void grad_viscosity(const AsmMesh& m, const double* u, const double* lam, int nq, long long ld, double* grad,
                    cudaStream_t s) {
    // columns per pass: as many as fit GQ_MAX and 96 KB of staging for the 8 warps
    const size_t per_col = sizeof(double) * 8 * m.d * m.nb;
    const int gq = (int)std::max<size_t>(1, std::min<size_t>(GQ_MAX, (96u << 10) / per_col));
    const size_t smem = per_col * gq;
    // a refused attribute surfaces as the launch error the caller checks
    if (smem > (48u << 10)) (void)cudaFuncSetAttribute(k_grad_nu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (int)std::min<long long>((m.nc + 7) / 8, 152LL * 16);
    k_grad_nu<<<grid, 256, smem, s>>>(m, u, lam, nq, ld, gq, grad);
}

void mass_apply_all(const AsmMesh& m, const double* lam, double scale, double* out, cudaStream_t s) {
    const long long n = (long long)m.d * m.nV;
    k_mass_all<<<(int)((n + 255) / 256), 256, 0, s>>>(m, lam, scale, out);
}

void cell_geometry(const AsmMesh& m, double* cg, cudaStream_t s) {
    k_cell_geometry<<<(m.nc + 127) / 128, 128, 0, s>>>(m, cg);
}

void set_list_caps(AsmMesh& m, int max_cells) {
    const long long cv = max_cells > 0 ? (long long)max_cells * m.nb : MAX_ROW;
    const long long cq = max_cells > 0 ? (long long)max_cells * m.nq : MAX_ROW;
    m.cap_v = (int)std::min<long long>(std::max<long long>(cv, 1), MAX_ROW);
    m.cap_q = (int)std::min<long long>(std::max<long long>(cq, 1), MAX_ROW);
}

void row_lengths(const AsmMesh& m, int* len, int* status, cudaStream_t s) {
    const int items = m.nVf + m.nQ;
    k_row_lengths<<<(items + WARPS - 1) / WARPS, WARPS * 32, WARPS * warp_list_bytes(m.cap_v, m.cap_q), s>>>(
        m, len, status);
}

void scan_rows(const int* len, int n, int* rp, int* tmp, cudaStream_t s) {
    const int nblk = (n + 1023) / 1024;
    k_scan_block<<<nblk, 1024, 0, s>>>(len, n, rp, tmp);
    k_scan_sums<<<1, 1, 0, s>>>(tmp, nblk);
    k_scan_add<<<(n + 255) / 256, 256, 0, s>>>(rp, n, tmp, nblk);
}

namespace {
__global__ void k_nc_count(long long m, const int* __restrict__ idx, int* __restrict__ cnt) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x)
        atomicAdd(cnt + idx[t], 1);
}
__global__ void k_nc_fill(long long m, const int* __restrict__ idx, const int* __restrict__ off, int* __restrict__ cur,
                          int* __restrict__ adj) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
        const int i = idx[t];
        adj[off[i] + atomicAdd(cur + i, 1)] = (int)t;
    }
}
// the fill's order within a list depends on the atomics: sort every list
__global__ void k_nc_sort(int n, const int* __restrict__ off, int* __restrict__ adj) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int* a = adj + off[i];
        const int len = off[i + 1] - off[i];
        for (int x = 1; x < len; ++x) {
            const int v = a[x];
            int y = x;
            for (; y > 0 && a[y - 1] > v; --y) a[y] = a[y - 1];
            a[y] = v;
        }
    }
}
}  // namespace

void node_cells(const int* cell_nodes, long long m, int n, int* off, int* adj, int* cnt, int* cur, int* tmp,
                cudaStream_t s) {
    if (n <= 0) return;
    cudaMemsetAsync(cnt, 0, sizeof(int) * n, s);
    cudaMemsetAsync(cur, 0, sizeof(int) * n, s);
    const int g = (int)std::min<long long>((m + 255) / 256, 152LL * 16);
    if (m > 0) k_nc_count<<<g, 256, 0, s>>>(m, cell_nodes, cnt);
    scan_rows(cnt, n, off, tmp, s);
    if (m > 0) k_nc_fill<<<g, 256, 0, s>>>(m, cell_nodes, off, cur, adj);
    k_nc_sort<<<(n + 255) / 256, 256, 0, s>>>(n, off, adj);
}

void fill_rows(const AsmMesh& m, const int* rp, int* ci, double* v, int* status, cudaStream_t s) {
    const int items = m.nVf + m.nQ;
    k_fill<<<(items + WARPS - 1) / WARPS, WARPS * 32, WARPS * warp_list_bytes(m.cap_v, m.cap_q), s>>>(
        m, rp, ci, v, status);
}

void load_vector(const AsmMesh& m, const double* f, const double* g, double inv_nu, double* b, cudaStream_t s) {
    const int rows = m.d * m.nVf + m.nQ;
    k_load<<<(rows + 127) / 128, 128, 0, s>>>(m, f, g, inv_nu, b);
}

}  // namespace sasm
