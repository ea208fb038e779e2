"""Taylor-Hood and Scott-Vogelius discretisations of stationary Stokes.
Oracle: test infrastructure.

Problem (Eq. 2.1 with all-Dirichlet velocity): -nu Laplace(u) + grad p = f,
-div u = 0, u = g_D on the boundary, p in L^2_0 (Sec. 2).  Weak form (Eq. 2.2):
a(u,v) = int nu grad u : grad v,  b(p,v) = -int p div v,  F(v) = int f . v.
Saddle-point matrix (Eq. 2.3): K = [A B^T; B 0].

DoF layout of the full (Dirichlet-included) vector: all velocity nodes of
component 0, then component 1 (then 2), then all pressure nodes.  The linear
system the solvers see keeps only the free DoFs (velocity nodes off the
boundary, every pressure node); Dirichlet DoFs are eliminated symmetrically
and their values lifted into the right-hand side.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import geometry, lagrange

TH, SV = 0, 1


class Space:
    """Scalar Lagrange space of degree k on a simplicial mesh (Sec. 2.1).

    continuous=True identifies nodes shared by neighbouring cells by the key
    {(vertex, alpha_vertex) : alpha_vertex > 0}; the set of those vertices is
    the mesh entity that owns the node.  continuous=False gives every cell its
    own nodes (the discontinuous P_{k-1}^disc pressure of Scott-Vogelius)."""

    def __init__(self, verts, cells, k, continuous=True):
        self.verts, self.cells, self.k = verts, np.asarray(cells), k
        self.d = self.cells.shape[1] - 1
        self.continuous = continuous
        alphas = lagrange.multi_indices(k, self.d)
        nb = len(alphas)
        nc = len(self.cells)
        self.nb = nb
        self.cell_nodes = np.empty((nc, nb), dtype=np.int64)
        keys, coords, entity = {}, [], []
        for ci, c in enumerate(self.cells.tolist()):
            for li, a in enumerate(alphas):
                if continuous:
                    key = tuple(sorted((c[i], a[i]) for i in range(self.d + 1) if a[i] > 0))
                else:
                    key = (ci, li)
                nid = keys.get(key)
                if nid is None:
                    nid = len(coords)
                    keys[key] = nid
                    x = sum(a[i] * verts[c[i]] for i in range(self.d + 1)) / max(k, 1)
                    coords.append(x)
                    if continuous:
                        entity.append(tuple(sorted(c[i] for i in range(self.d + 1) if a[i] > 0)))
                    else:
                        entity.append(tuple(sorted(c)))
                self.cell_nodes[ci, li] = nid
        self.coords = np.asarray(coords)
        self.entity = entity
        self.n = len(coords)
        self.keys = keys

    def boundary_mask(self):
        """True for nodes whose owning entity lies on the boundary."""
        bnd = geometry.boundary_entities(self.cells)
        return np.array([e in bnd for e in self.entity], dtype=bool)


@dataclass
class Discretization:
    """Assembled Stokes operator on one mesh (Eq. 2.3)."""
    verts: np.ndarray
    cells: np.ndarray
    family: int
    k: int
    V: Space
    Q: Space
    Kfull: sp.csr_matrix
    Mv: sp.csr_matrix           # scalar P_k mass matrix (all nodes)
    p_integrals: np.ndarray     # int psi_j for every pressure node
    dirichlet: np.ndarray       # bool over the full DoF vector
    free: np.ndarray            # indices of free DoFs in the full vector
    K: sp.csr_matrix            # free-free block

    @property
    def d(self):
        return self.V.d

    @property
    def n_full(self):
        return self.d * self.V.n + self.Q.n

    @property
    def n_free(self):
        return len(self.free)

    def pressure_mask_free(self):
        return self.free >= self.d * self.V.n

    def dof_coords_full(self):
        """(coordinates, component) of every full DoF; component d = pressure."""
        xs = [self.V.coords] * self.d + [self.Q.coords]
        comp = np.concatenate([np.full(self.V.n, c) for c in range(self.d)] + [np.full(self.Q.n, self.d)])
        return np.concatenate(xs, axis=0), comp


def element_matrices(verts, cells, k, kq, d):
    """Per-cell scalar stiffness S, mass M (P_k x P_k) and divergence coupling
    C[c, q, b, comp] = -int psi_q d(phi_b)/dx_comp  (P_kq pressure), computed
    with a quadrature exact for degree 2k on affine simplices."""
    lam, w = lagrange.quadrature(d, 2 * k)
    phi = lagrange.basis(k, d, lam)              # [nq, nb]
    dphi = lagrange.basis_dlam(k, d, lam)        # [nq, nb, d+1]
    psi = lagrange.basis(kq, d, lam)             # [nq, np]
    G, vol = lagrange.barycentric_gradients(verts, cells)
    nc = len(cells)
    nb, npp = phi.shape[1], psi.shape[1]
    S = np.empty((nc, nb, nb))
    M = np.empty((nc, nb, nb))
    C = np.empty((nc, npp, nb, d))
    Mref = np.einsum("q,qa,qb->ab", w, phi, phi)
    for s in range(0, nc, 2048):
        e = slice(s, min(nc, s + 2048))
        gphi = np.einsum("qbi,cid->cqbd", dphi, G[e])
        S[e] = vol[e, None, None] * np.einsum("q,cqad,cqbd->cab", w, gphi, gphi)
        C[e] = -vol[e, None, None, None] * np.einsum("q,qp,cqbd->cpbd", w, psi, gphi)
        M[e] = vol[e, None, None] * Mref[None]
    return S, M, C, vol


def discretize(verts, cells, family, k, nu_cells=None):
    """Assemble K = [nu A, B^T; B, 0] for TH P_k/P_{k-1} or SV
    P_k/P_{k-1}^disc (Sec. 2.1, Eq. 2.3); A is the vector Laplacian, B the
    negative divergence.  nu_cells scales A cell-wise (default 1)."""
    verts = np.asarray(verts, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64)
    d = cells.shape[1] - 1
    V = Space(verts, cells, k, continuous=True)
    Q = Space(verts, cells, k - 1, continuous=(family == TH))
    S, M, C, vol = element_matrices(verts, cells, k, k - 1, d)
    nu = np.ones(len(cells)) if nu_cells is None else np.asarray(nu_cells, dtype=np.float64)
    nV, nQ = V.n, Q.n
    N = d * nV + nQ
    rows, cols, vals = [], [], []
    cn, qn = V.cell_nodes, Q.cell_nodes
    nb, npp = cn.shape[1], qn.shape[1]
    Ar = np.repeat(cn[:, :, None], nb, axis=2)
    Ac = np.repeat(cn[:, None, :], nb, axis=1)
    Av = nu[:, None, None] * S
    for c in range(d):
        rows.append((c * nV + Ar).ravel()); cols.append((c * nV + Ac).ravel()); vals.append(Av.ravel())
    Br = np.repeat(qn[:, :, None], nb, axis=2)
    Bc = np.repeat(cn[:, None, :], npp, axis=1)
    for c in range(d):
        r = (d * nV + Br).ravel()
        cc = (c * nV + Bc).ravel()
        v = C[:, :, :, c].ravel()
        rows += [r, cc]; cols += [cc, r]; vals += [v, v]
    Kfull = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
    Kfull.sum_duplicates()
    Mv = sp.csr_matrix((M.ravel(), (Ar.ravel(), Ac.ravel())), shape=(nV, nV))
    Mv.sum_duplicates()
    # int psi_j: the pressure basis integrals (for the zero-mean constraint)
    lam, w = lagrange.quadrature(d, k)
    psi = lagrange.basis(k - 1, d, lam)
    pint_loc = vol[:, None] * (w @ psi)[None, :]
    p_integrals = np.bincount(qn.ravel(), weights=pint_loc.ravel(), minlength=nQ)
    bmask = V.boundary_mask()
    dirichlet = np.concatenate([bmask] * d + [np.zeros(nQ, dtype=bool)])
    free = np.flatnonzero(~dirichlet)
    K = Kfull[free][:, free].tocsr()
    return Discretization(verts, cells, family, k, V, Q, Kfull, Mv, p_integrals, dirichlet, free, K)


def load_vector(disc: Discretization, f_nodal, g_nodal=None):
    """Free-DoF right-hand side b: F = int f.v with f given by nodal values
    (F_c = M_v f_c exactly), minus the lifting K[free, D] g_D of the Dirichlet
    data (g_nodal [d, nV], only boundary nodes used); pressure rows get
    -B[:, D] g_D.  The component of b along the pressure null vector
    (constants, Sec. 2: p is fixed only up to a constant) is removed so that
    the singular system is consistent."""
    d, nV = disc.d, disc.V.n
    F = np.zeros(disc.n_full)
    f_nodal = np.asarray(f_nodal, dtype=np.float64).reshape(d, nV)
    for c in range(d):
        F[c * nV:(c + 1) * nV] = disc.Mv @ f_nodal[c]
    xD = np.zeros(disc.n_full)
    if g_nodal is not None:
        g = np.asarray(g_nodal, dtype=np.float64).reshape(d, nV)
        xD[:d * nV] = g.ravel()
        xD[~disc.dirichlet] = 0.0
    b = (F - disc.Kfull @ xD)[disc.free]
    pm = disc.pressure_mask_free()
    b[pm] -= b[pm].mean()
    return b, xD


def expand(disc: Discretization, x_free, xD):
    """Full vector (velocity incl. boundary values, pressure) from free DoFs."""
    x = xD.copy()
    x[disc.free] = x_free
    return x


def zero_mean_pressure(disc: Discretization, x_full):
    """Shift p so that int p = 0 (the L^2_0 normalisation of Sec. 2)."""
    d, nV = disc.d, disc.V.n
    p = x_full[d * nV:]
    c = (disc.p_integrals @ p) / disc.p_integrals.sum()
    out = x_full.copy()
    out[d * nV:] = p - c
    return out


def direct_solve(disc: Discretization, b, refine=1):
    """Sparse direct solve of the free system bordered by the zero-mean
    pressure constraint (Sec. 2: p in L^2_0), followed by `refine` steps of
    iterative refinement with the same LU factors (x += LU^-1 (rhs - Kb x),
    residual in FP64).  A plain sparse LU leaves an error of about
    eps * cond(Kb) in the solution (1e-10 relative in the pressure of the
    P4/P3 32x32 problem); one refinement step brings it to the rounding level
    of the discrete solution."""
    import scipy.sparse.linalg as spla
    n = disc.n_free
    c = np.zeros(n)
    pm = disc.pressure_mask_free()
    c[pm] = disc.p_integrals[disc.free[pm] - disc.d * disc.V.n]
    Kb = sp.bmat([[disc.K, sp.csr_matrix(c[:, None])], [sp.csr_matrix(c[None, :]), None]]).tocsc()
    rhs = np.concatenate([b, [0.0]])
    lu = spla.splu(Kb)
    x = lu.solve(rhs)
    for _ in range(refine):
        x = x + lu.solve(rhs - Kb @ x)
    return x[:n]


def l2_errors(disc: Discretization, x_full, u_exact, p_exact, qdeg=None):
    """||u - u_h||_L2 and ||p - p_h||_L2 by quadrature on every cell."""
    d, k = disc.d, disc.k
    qdeg = qdeg or 2 * k + 4
    lam, w = lagrange.quadrature(d, qdeg)
    phi = lagrange.basis(k, d, lam)
    psi = lagrange.basis(k - 1, d, lam)
    verts, cells = disc.verts, disc.cells
    _, vol = lagrange.barycentric_gradients(verts, cells)
    X = np.einsum("qi,cid->cqd", lam, verts[cells])
    nV = disc.V.n
    U = x_full[:d * nV].reshape(d, nV)
    P = x_full[d * nV:]
    uh = np.stack([np.einsum("qb,cb->cq", phi, U[c][disc.V.cell_nodes]) for c in range(d)], axis=-1)
    ph = np.einsum("qb,cb->cq", psi, P[disc.Q.cell_nodes])
    eu = ((u_exact(X) - uh) ** 2).sum(-1)
    ep = (p_exact(X) - ph) ** 2
    return np.sqrt((vol[:, None] * w[None] * eu).sum()), np.sqrt((vol[:, None] * w[None] * ep).sum())
