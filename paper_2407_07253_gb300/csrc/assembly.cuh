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
};

// Per-cell factors of the affine map x = x_0 + J xi, computed once per level:
//   cg[0]                 |det J|
//   cg[1 + a d + b]       nu_e |det J| sum_c Jinv[a][c] Jinv[b][c]   (stiffness)
//   cg[1 + d d + a d + c] -|det J| Jinv[a][c]                        (divergence)
constexpr int CG_STRIDE = 20;
void cell_geometry(const AsmMesh& m, double* cg, cudaStream_t s);

constexpr int MAX_ROW = 1024;          // neighbours of one node (per kind)

// Pass 1: row lengths.  len[r] for r < d*nVf + nQ.
void row_lengths(const AsmMesh& m, int* len, int* status, cudaStream_t s);
// Exclusive scan of len into rp[0..n] (rp[n] = total); tmp holds
// ceil(n / 1024) + 1 ints.
void scan_rows(const int* len, int n, int* rp, int* tmp, cudaStream_t s);
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

}  // namespace sasm
