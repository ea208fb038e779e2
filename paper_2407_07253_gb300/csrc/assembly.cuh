// Device assembly of K = [nu A, B^T; B, 0] (Eq. 2.3) on the free DoFs, and
// the matrix-free load vector F = M f with the Dirichlet lifting
// -K[free, D] g (Sec. 2), from the mesh, the DoF maps and the exact
// reference tensors of the Lagrange pair.
//
// Rows follow the library's free order: the d velocity components of every
// free velocity node, then every pressure node.  A row's columns are its
// neighbours in order of first appearance over the node's incident cells
// (cells in increasing index, local nodes in element order), velocity
// columns first, so every row is reproducible bit for bit; rows are not
// sorted by column.
#pragma once
#include <cuda_runtime.h>

namespace sasm {

struct AsmMesh {
    int d, nc, nb, nq;                 // dimension, cells, velocity / pressure nodes per cell
    int nV, nQ, nVf;                   // velocity nodes, pressure nodes, free velocity nodes
    const double* X;                   // [nv][d] vertex coordinates
    const int* C;                      // [nc][d+1] cell vertices
    const int* vcell;                  // [nc][nb] velocity node ids
    const int* qcell;                  // [nc][nq] pressure node ids
    const int* vfree;                  // [nV] free index or -1
    const int* vrow;                   // [nVf] free index -> velocity node
    const int* voff; const int* vadj;  // velocity node -> cell*nb + local
    const int* qoff; const int* qadj;  // pressure node -> cell*nq + local
    const double* nu;                  // [nc] or nullptr
    const double* S;                   // [d][d][nb][nb] reference stiffness tensors
    const double* Cq;                  // [d][nq][nb] int psi_p d(phi_j)/dxi_a
    const double* M;                   // [nb][nb] reference mass matrix
    const double* cg;                  // [nc][CG_STRIDE] per-cell factors (cell_geometry)
    int cap_v, cap_q;                  // list capacity per node (velocity / pressure neighbours):
                                       // set by set_list_caps
};

// Per-cell factors of the affine map x = x_0 + J xi, computed once per level:
//   cg[0]                 |det J|
//   cg[1 + a d + b]       nu_e |det J| sum_c Jinv[a][c] Jinv[b][c]   (stiffness)
//   cg[1 + d d + a d + c] -|det J| Jinv[a][c]                        (divergence)
constexpr int CG_STRIDE = 20;
void cell_geometry(const AsmMesh& m, double* cg, cudaStream_t s);

constexpr int MAX_ROW = 1024;          // neighbours of one node (per kind)

// List capacities for row_lengths / fill_rows: a node in at most max_cells
// cells has at most max_cells * nb velocity and max_cells * nq pressure
// neighbours (capped at MAX_ROW; max_cells <= 0: MAX_ROW).  A row that does
// not fit sets the status word.
void set_list_caps(AsmMesh& m, int max_cells);

// Pass 1: row lengths.  len[r] for r < d*nVf + nQ.
void row_lengths(const AsmMesh& m, int* len, int* status, cudaStream_t s);
// Exclusive scan of len into rp[0..n] (rp[n] = total); tmp holds
// ceil(n / 1024) + 1 ints.
void scan_rows(const int* len, int n, int* rp, int* tmp, cudaStream_t s);
// Incidence lists of a space's nodes: adj[off[i] .. off[i+1]) holds the
// positions t = e * per_cell + l of node i in cell_nodes[0 .. m), in
// increasing order (so the incident cells in increasing index).  cnt and cur
// hold n ints, tmp ceil(n / 1024) + 1; off n + 1, adj m.
void node_cells(const int* cell_nodes, long long m, int n, int* off, int* adj, int* cnt, int* cur, int* tmp,
                cudaStream_t s);
// Pass 2: columns and values.
void fill_rows(const AsmMesh& m, const int* rp, int* ci, double* v, int* status, cudaStream_t s);
// b[r] = (M f)(row r) / nu_const on velocity rows, 0 on pressure rows, minus
// K[r, D] g for Dirichlet data g ([d][nV], only boundary nodes read; may be
// nullptr).  f is [d][nV].
void load_vector(const AsmMesh& m, const double* f, const double* g, double inv_nu, double* b, cudaStream_t s);

// Adjoint pieces (the discrete adjoint of the solve):
// grad[e] = -sum_q sum_c lambda_q,c[e]^T A_e u_q,c[e] for every cell, A_e
// the unit-viscosity stiffness of cell e; u and lambda are nq [d][nV] nodal
// fields ld doubles apart (u with its boundary values, lambda zero on the
// boundary).
void grad_viscosity(const AsmMesh& m, const double* u, const double* lam, int nq, long long ld, double* grad,
                    cudaStream_t s);
// out[c][i] = scale (M lambda_c)[i] for every velocity node i.
void mass_apply_all(const AsmMesh& m, const double* lam, double scale, double* out, cudaStream_t s);

// ---- finite-element interpolation P between consecutive levels (Sec. 3.1)
// built on the device: row i of the scalar P holds the coarse basis
// functions evaluated at fine node i, located in the coarse cell that
// contains (or is) the cell owning it; entries with |v| <= 1e-14 (exact
// lattice zeros) are dropped and a row's columns are sorted.
struct InterpSpace {
    int nb = 0;                  // nodes per cell
    const int* cell = nullptr;   // [nc][nb] node ids
    const int* off = nullptr;    // fine side: node -> (cell * nb + local) adjacency,
    const int* adj = nullptr;    //   cells in increasing order (the first one owns the node)
    const int* free = nullptr;   // node -> free index or -1; nullptr: every node free, index = node
};
struct InterpGeom {
    int d = 0;
    int nested = 0;              // 0: same mesh (table), 1: coarse mesh = parent of the fine mesh
    const double* tab = nullptr; // same mesh: [nb_f][nb_c] coarse basis at the fine lattice points
    const int* parent = nullptr; // nested: fine cell -> coarse cell
    const double* Xf = nullptr; const int* Cf = nullptr;   // nested: fine mesh
    const double* Xc = nullptr; const int* Cc = nullptr;   // nested: coarse mesh
    int kf = 0;                  // nested: fine degree; alpha_f [nb_f][4] its lattice multi-indices
    const int* alpha_f = nullptr;
    int nm = 0;                  // nested: coarse basis as monomials, mono [nm][3] exponents,
    const int* mono = nullptr;   //   coef [nb_c][nm]
    const double* coef = nullptr;
};
constexpr int INTERP_MAX_NB = 64;   // coarse nodes per cell handled on the device
// Scalar rows for the nrows fine nodes rows[0..nrows) (rows == nullptr: node
// = row), at most nb_c entries each, in fixed slots: cnt[row],
// col[row * nb_c + t] (coarse free index), val[row * nb_c + t].
void interp_rows(const InterpGeom& g, const InterpSpace& fine, const InterpSpace& coarse, int nrows, const int* rows,
                 int* cnt, int* col, double* val, cudaStream_t s);
// Monolithic P = blockdiag(P_V, ..., P_V, P_Q) on the free DoFs from the
// scalar slots (velocity rows over the fine free velocity nodes, pressure
// rows over the fine pressure nodes): len[r] for r < d nVf + nQf.
void interp_lengths(int d, int nVf, int nQf, const int* cntV, const int* cntQ, int* len, cudaStream_t s);
void interp_fill(int d, int nVf, int nQf, int nVf_c, int sV, int sQ, const int* cntV, const int* colV,
                 const double* valV, const int* cntQ, const int* colQ, const double* valQ, const int* rp, int* ci,
                 double* v, cudaStream_t s);
// R = P^T: counts, (scan), fill, then each row sorted by column: a
// deterministic transpose.  cnt / cur hold ncol ints each (zeroed here).
void transpose_count(int nr, const int* rp, const int* ci, int ncol, int* cnt, cudaStream_t s);
void transpose_fill(int nr, const int* rp, const int* ci, const double* v, int ncol, const int* rrp, int* cur,
                    int* rci, double* rv, cudaStream_t s);
void sort_rows(int nr, const int* rp, int* ci, double* v, cudaStream_t s);
void to_float(long long n, const double* x, float* y, cudaStream_t s);

}  // namespace sasm
