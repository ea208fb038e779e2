"""Full-block-factorisation preconditioner FBF(phMG) for Scott-Vogelius
(Eq. fbf, Fig. afbf_solver; the relaxation of Sec. 3.3).  Oracle: test
infrastructure.

For K = [A B^T; B 0] (free DoFs), Eq. fbf composes
    P^-1 = [I  -A~^-1 B^T; 0  I] diag(A~^-1, S~^-1) [I  0; -B A~^-1  I],
so that for r = (r_u, r_p)
    a   = A~^-1 r_u
    z_p = S~^-1 (r_p - B a)
    z_u = A~^-1 (r_u - B^T z_p)        (A~^-1 is linear: a fixed V-cycle)
with
  * A~^-1: one phMG V-cycle on the velocity block.  A is the vector
    Laplacian int nu grad u : grad v, block diagonal over the d components
    with the scalar nu-weighted stiffness A_s in each block, so A~^-1 is the
    scalar phMG V-cycle applied to every component.  Its hierarchy is that of
    the monolithic solver (p-levels on the finest, Alfeld-refined mesh, then
    h-levels of the last degree on the nested meshes, exact coarsest solve);
    its relaxation is Chebyshev(nu) around one additive Schwarz sweep over
    ASMStarPC patches: per mesh vertex v, the DoFs on the open star of v (the
    vertex, and the edges, faces and cells containing it; not the closure).
  * S~^-1: the inverse of the block-diagonal discontinuous pressure mass
    matrix, spectrally equivalent to the inverse Schur complement.

Readings of points the paper leaves open: the Schur complement of K is
S = -B A^-1 B^T, which is negative definite, so S~^-1 = -diag_e(nu_e M_p,e^-1), with nu_e
the cell viscosity (the standard scaling for a variable viscosity; 1 for
constant unit viscosity).  The partition-of-unity weights, the Chebyshev
interval and the Arnoldi estimate follow oracle.multigrid.
"""
from types import SimpleNamespace

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import geometry, lagrange, multigrid, rng, stokes


def scalar_stiffness(verts, cells, k, nu_cells=None):
    """(A_s on all nodes, the Space) for the scalar P_k stiffness
    sum_e nu_e int grad phi_i . grad phi_j."""
    V = stokes.Space(verts, cells, k, continuous=True)
    d = V.d
    S, _, _, _ = stokes.element_matrices(verts, cells, k, k - 1, d)
    nu = np.ones(len(cells)) if nu_cells is None else np.asarray(nu_cells, dtype=np.float64)
    cn = V.cell_nodes
    nb = cn.shape[1]
    rows = np.repeat(cn[:, :, None], nb, axis=2).ravel()
    cols = np.repeat(cn[:, None, :], nb, axis=1).ravel()
    A = sp.csr_matrix(((nu[:, None, None] * S).ravel(), (rows, cols)), shape=(V.n, V.n))
    A.sum_duplicates()
    return A, V


def star_patches(V: stokes.Space, free):
    """ASMStarPC patches: for every mesh vertex v the free nodes whose owning
    entity contains v (the open star of v), as sorted free indices."""
    node_to_free = -np.ones(V.n, dtype=np.int64)
    node_to_free[free] = np.arange(len(free))
    by_vertex = {}
    for node, ent in enumerate(V.entity):
        f = node_to_free[node]
        if f < 0:
            continue
        for v in ent:
            by_vertex.setdefault(v, []).append(f)
    return [np.array(sorted(by_vertex[v]), dtype=np.int64) for v in sorted(by_vertex)]


class VelocityHierarchy(multigrid.Hierarchy):
    """The scalar phMG hierarchy of A~^-1 (one velocity component).  Levels
    reuse multigrid.Hierarchy's cycle: each carries `disc.K` = A_s on the free
    nodes, ASMStarPC patches, P, R and lambda_max."""

    def __init__(self, verts, cells, n_refine, schedule, barycentric=True, nu_cells=None,
                 opts: multigrid.Options = None, lmax=None):
        self.opts = opts or multigrid.Options()
        meshes, parents = geometry.hierarchy(verts, cells, n_refine, barycentric)
        self.meshes, self.parents = meshes, parents
        nus = [None if nu_cells is None else np.asarray(nu_cells, dtype=np.float64)]
        for mi in range(len(meshes) - 1):
            if nus[-1] is None:
                nus.append(None)
                continue
            par = parents[mi]
            s = np.bincount(par, weights=nus[-1], minlength=len(meshes[mi + 1][1]))
            cnt = np.bincount(par, minlength=len(meshes[mi + 1][1]))
            nus.append(s / cnt)
        specs = [(0, deg, "p") for deg in schedule[:-1]]
        specs += [(mi, schedule[-1], "h" if mi < len(meshes) - 1 else "coarse") for mi in range(len(meshes))]
        self.levels = []
        for mi, deg, kind in specs:
            A, V = scalar_stiffness(*meshes[mi], deg, nus[mi])
            free = np.flatnonzero(~V.boundary_mask())
            disc = SimpleNamespace(K=A[free][:, free].tocsr(), n_free=len(free), V=V, free=free,
                                   verts=meshes[mi][0], cells=meshes[mi][1])
            self.levels.append(multigrid.Level(disc, kind, mi))
        for i in range(len(self.levels) - 1):
            fine, coarse = self.levels[i], self.levels[i + 1]
            f2c = (np.arange(len(fine.disc.cells)) if fine.mesh_index == coarse.mesh_index
                   else parents[fine.mesh_index])
            PV = multigrid.scalar_interpolation(coarse.disc.V, fine.disc.V, f2c)
            fine.P = PV[fine.disc.free][:, coarse.disc.free].tocsr()
            fine.R = fine.P.T.tocsr()
        for i, L in enumerate(self.levels[:-1]):
            L.asm = multigrid.ASM(L.disc.K, star_patches(L.disc.V, L.disc.free))
            if lmax is not None and lmax[i] is not None:
                L.lmax = float(lmax[i])
            else:
                v0 = rng.uniform_pm1(self.opts.eig_seed, i, np.arange(L.disc.n_free))
                L.lmax = multigrid.arnoldi_lmax(L.disc.K, L.asm.apply, v0, self.opts.eig_steps)
        self.coarse_lu = sla.lu_factor(self.levels[-1].disc.K.toarray())

    def coarse_solve(self, r):
        """Exact solve with the coarsest A_s (Dirichlet, so nonsingular)."""
        return sla.lu_solve(self.coarse_lu, r)


def pressure_mass_blocks(disc: stokes.Discretization):
    """Per-cell blocks M_p,e[a, b] = int_e psi_a psi_b of the discontinuous
    pressure space (exact quadrature), with the cells' pressure nodes."""
    d, kq = disc.d, disc.k - 1
    lam, w = lagrange.quadrature(d, 2 * kq)
    psi = lagrange.basis(kq, d, lam)
    Mref = np.einsum("q,qa,qb->ab", w, psi, psi)
    _, vol = lagrange.barycentric_gradients(disc.verts, disc.cells)
    return vol[:, None, None] * Mref[None], disc.Q.cell_nodes


class FBF:
    """P^-1 of Eq. fbf on the free DoFs of an SV discretisation (velocity
    components blocked, then pressure, as stokes.Discretization orders them)."""

    def __init__(self, disc: stokes.Discretization, vh: VelocityHierarchy, nu_cells=None, a_solve=None,
                 s_solve=None):
        assert not disc.Q.continuous, "FBF uses the block-diagonal (discontinuous) pressure mass matrix"
        self.disc, self.vh = disc, vh
        d, nV = disc.d, disc.V.n
        self.nu_free = int(np.sum(disc.free < d * nV))
        self.nvf = self.nu_free // d
        K = disc.K.tocsr()
        self.B = K[self.nu_free:, :self.nu_free].tocsr()
        self.BT = K[:self.nu_free, self.nu_free:].tocsr()
        nu = np.ones(len(disc.cells)) if nu_cells is None else np.asarray(nu_cells, dtype=np.float64)
        Mp, qn = pressure_mass_blocks(disc)
        self.qn = qn
        self.Sinv_blocks = -nu[:, None, None] * np.linalg.inv(Mp)
        self._a = a_solve or self._vcycle_components
        self._s = s_solve or self._schur_inverse

    def _vcycle_components(self, ru):
        return np.concatenate([self.vh.vcycle(ru[c * self.nvf:(c + 1) * self.nvf]) for c in range(self.disc.d)])

    def _schur_inverse(self, yp):
        z = np.zeros_like(yp)
        for e in range(len(self.qn)):
            q = self.qn[e]
            z[q] = self.Sinv_blocks[e] @ yp[q]
        return z

    def apply(self, r):
        r = np.asarray(r, dtype=np.float64)
        ru, rp = r[:self.nu_free], r[self.nu_free:]
        a = self._a(ru)
        zp = self._s(rp - self.B @ a)
        zu = self._a(ru - self.BT @ zp)
        return np.concatenate([zu, zp])


def solve(fbf: FBF, f_nodal, g_nodal=None, tol=1e-8, restart=30, maxit=1000):
    """stokes_solve with FBF(phMG): load vector, lifting, FGMRES right-
    preconditioned by Eq. fbf, zero-mean pressure."""
    disc = fbf.disc
    b, xD = stokes.load_vector(disc, f_nodal, g_nodal)
    x, its, hist = multigrid.fgmres(disc.K, b, fbf.apply, tol, restart, maxit)
    full = stokes.zero_mean_pressure(disc, stokes.expand(disc, x, xD))
    return full, its, hist
