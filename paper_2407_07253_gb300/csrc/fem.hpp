// Host-side finite-element setup of the phMG hierarchy: nested simplicial
// meshes (uniform R_u and Alfeld R_b refinement, Fig. 1), equispaced
// Lagrange P_k spaces (Sec. 2.1), assembly of K = [nu A, B^T; B, 0]
// (Eq. 2.3) into CSR on the free DoFs, finite-element interpolation P and
// R = P^T (Sec. 3.1), and the Vanka-star patch index sets (Sec. 3.4, Fig. 5).
// Everything numeric that runs per V-cycle lives in the CUDA kernels; this
// file only produces the index structures and matrix values that the device
// setup consumes.
#pragma once
#include <array>
#include <cstdint>
#include <functional>
#include <string>
#include <memory>
#include <utility>
#include <vector>

namespace sfem {

// std::vector storage whose resize() leaves trivially constructible
// elements uninitialised, so that large arrays are first touched (and their
// pages faulted in) by the parallel loops that fill them.
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
    template <class U>
    struct rebind { using other = DefaultInitAlloc<U>; };
    DefaultInitAlloc() = default;
    template <class U>
    DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
    template <class U>
    void construct(U* p) noexcept { ::new ((void*)p) U; }
    template <class U, class... A>
    void construct(U* p, A&&... a) { ::new ((void*)p) U(std::forward<A>(a)...); }
};
template <class T>
using fvec = std::vector<T, DefaultInitAlloc<T>>;

struct Mesh {
    int d = 0, nv = 0, nc = 0;
    std::vector<double> X;   // [nv][d]
    std::vector<int> C;      // [nc][d+1]
};

Mesh refine_uniform(const Mesh& m, std::vector<int>& parent);
Mesh refine_alfeld(const Mesh& m, std::vector<int>& parent);

// Lagrange element of degree k on the reference d-simplex with the
// equispaced lattice nodes xi = (alpha_1, ..., alpha_d) / k.  The basis is
// held in Bernstein form (bcoef: phi_i = sum_b bcoef[i][b] B_b, b in the
// order of alpha), which eval and the reference tensors use, and expanded
// in monomials (coef, from inverting the Vandermonde matrix of the nodes)
// for the device kernel that evaluates the coarse basis of the h-transfers
// (P2 in every phMG hierarchy, where the expansion is exact; it loses
// digits at high degree).
struct RefElement {
    int d = 0, k = 0, nb = 0, nm = 0;
    std::vector<std::array<int, 4>> alpha;   // [nb] barycentric multi-index, alpha[0] = k - sum
    std::vector<std::array<int, 3>> mono;    // [nm] exponents
    std::vector<double> coef;                // [nb][nm]
    std::vector<double> bcoef;               // [nb][nb]
    void init(int d, int k);
    void eval(const double* xi, double* out) const;   // out[nb]
};

// Reference tensors of one (velocity degree k, pressure degree kq) pair on
// the reference simplex (volume 1/d!), from the Lagrange basis in Bernstein
// form and the closed-form integrals of Bernstein products, summed with
// compensated arithmetic: accurate to a few units of the last place up to
// k = 10 (a monomial expansion loses up to five digits there).
struct RefTensors {
    int d = 0, nb = 0, nq = 0;
    std::vector<double> S;     // [d][d][nb][nb]   int dphi_i/dxi_a dphi_j/dxi_b
    std::vector<double> Cq;    // [d][nq][nb]      int psi_p dphi_j/dxi_a
    std::vector<double> M;     // [nb][nb]         int phi_i phi_j
    std::vector<double> qint;  // [nq]             int psi_p
    void init(const RefElement& v, const RefElement& q);
};

struct CSR {
    int nr = 0, ncol = 0;
    fvec<int> rp, ci;
    fvec<double> v;
    long long nnz() const { return (long long)ci.size(); }
};
CSR transpose(const CSR& a);

struct Space {
    int d = 0, k = 0, nb = 0, n = 0;
    bool continuous = true;
    std::vector<int> cell_nodes;               // [nc][nb]
    fvec<double> X;                            // [n][d]
    fvec<unsigned char> boundary;              // [n]
    fvec<std::array<int, 4>> support;          // [n] vertices of the owning entity (-1 padded)
    fvec<int> owner_cell;                      // [n] a cell containing the node
    fvec<int> owner_local;                     // [n] the node's local index in owner_cell
};

struct Level {
    int d = 0, family = 0, k = 0, mesh_index = 0;
    bool p_level = false;
    Space V, Q;
    std::vector<int> vfree;    // velocity node -> free node index or -1
    int nVf = 0, nQ = 0, n_free = 0;
    CSR K;                     // free x free
    CSR KfD;                   // free rows x full velocity DoFs (Dirichlet columns only)
    CSR Mv;                    // scalar velocity mass matrix on all nodes
    std::vector<double> pint;  // int psi_j for every pressure node
    CSR P, R;                  // interpolation from level+1 (free x free) and its transpose
    std::vector<int> patch_off, patch_dofs;   // Vanka-star patches (free DoF indices)
    std::vector<int> patch_nv;                // velocity nodes per component of each patch:
                                              // a patch lists d blocks of n_v velocity DoFs
                                              // (same nodes per component), then n_p pressures
    std::vector<double> cell_center;          // [nc][d]
    // what a device assembly needs: node -> (cell * nb + local) adjacency,
    // the reference tensors and the cell viscosities
    std::vector<int> voff, vadj, qoff, qadj;
    int max_cells = 0;                        // most cells around one vertex of the mesh: no
                                              // node lies in more cells than that
    RefTensors RT;
    std::vector<double> nu_cells;
    bool host_matrices = true;                // K (and on level 0 Mv, KfD) assembled here
};

struct HierarchySpec {
    int family = 0, k = 2;
    std::vector<int> schedule;   // velocity degrees of the p-levels + the hMG degree
    int n_refine = 0;
    bool barycentric = false;
    bool device_assembly = false;             // leave K of all but the coarsest level to the device
    // order of construction (and of the per-level callbacks): false = finest
    // to coarsest; true = the coarsest level first (its device factorisation
    // is a long chain of small steps that then runs while the host builds the
    // other levels), then finest to coarsest
    bool coarsest_first = false;
    // with coarsest_first: the coarsest level is built on a host thread of
    // its own (its loops run inline there, off the shared pool) while this
    // thread builds the others, finest to coarsest; the per-level callbacks
    // then come from two threads and must be thread-safe
    bool coarsest_thread = false;
    bool skip_patches = false;                // no Vanka patches (a hierarchy wanted for its operators)
    bool device_assembly_finest_only = false; // with device_assembly: only level 0 on the device
    bool device_transfers = false;            // leave P and R to the device (no host transfers)
};

struct Hierarchy {
    std::vector<Mesh> meshes;                 // [0] = finest
    std::vector<std::vector<int>> parents;    // parents[i]: cells of meshes[i] -> meshes[i+1]
    std::vector<Level> levels;
    double t_mesh_ms = 0, t_assembly_ms = 0;
    double t_spaces_ms = 0, t_matrices_ms = 0, t_patches_ms = 0, t_transfers_ms = 0, t_callbacks_ms = 0;
};

// The scalar hierarchy of one velocity component of a host-assembled Stokes
// hierarchy S (the velocity block of Eq. 2.3 is the vector Laplacian, block
// diagonal over the components with one scalar stiffness A_s): per level the
// velocity space and free nodes, K = A_s (the component-0 block of S's K),
// P and R = the component-0 blocks of S's transfers, and ASMStarPC patches,
// the free nodes on the open star of every mesh vertex (the nodes whose
// owning entity contains the vertex).  No pressure.  A level of S without a
// host K (device assembly) gets an empty K and host_matrices = false: its
// velocity block is then extracted on the device.
void velocity_hierarchy(Hierarchy& S, Hierarchy& A);

// Mass matrix [nb][nb] of the degree-k Lagrange element on the reference
// d-simplex (exact).
std::vector<double> reference_mass(int d, int k);

// Build the whole host hierarchy; throws std::runtime_error on invalid input.
// on_level(l, stage), if given, runs twice per level: stage 0 once its
// spaces and operator data exist, stage 1 once its patches exist too (levels
// in the order that spec.coarsest_first selects; the transfers are built
// after every level), so the caller can start device work on each part
// while the host continues.
void build_hierarchy(const Mesh& coarse, const HierarchySpec& spec, const double* nu_cell,
                     Hierarchy& H, const std::function<void(int, int)>& on_level = {});

int num_threads();

// The degree-k Lagrange element on the reference d-simplex, computed once per
// process and kept (references stay valid).
const RefElement& reference_element(int d, int k);

// For idx[0..m) with values in [0, n): off[0..n] and pos[0..m) list, for
// every value, the positions q where it occurs, in increasing order
// (parallel counting sort).
void invert_index(const int* idx, long long m, int n, std::vector<int>& off, std::vector<int>& pos);

// memcpy split over the host worker pool
void parallel_copy(void* dst, const void* src, size_t bytes);

}  // namespace sfem
