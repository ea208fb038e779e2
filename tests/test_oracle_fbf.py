"""Pins of the FBF(phMG) oracle (oracle/fbf.py; Eq. fbf, Sec. 3.3).

  * Eq. fbf with exact blocks (A~ = A, S~ = -B A^-1 B^T) is the exact inverse
    of a nonsingular saddle matrix: P^-1 K = I.  A sign or ordering slip in the
    composition fails this.
  * ASMStarPC patches equal the open vertex stars defined geometrically: a
    node belongs to star(v) iff its barycentric coordinate of v is positive in
    a cell that contains both (independent of the entity bookkeeping).
  * The discontinuous pressure mass blocks: their entries sum to the cell
    volume (int 1 = |e|), and the assembled global mass matrix of the SV
    pressure space is exactly their block diagonal.
  * The scalar phMG V-cycle of A~^-1 contracts the error of A_s x = b.
  * FGMRES with FBF reaches the direct solution of the SV system, in fewer
    iterations than without preconditioning.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fbf, geometry, lagrange, multigrid, stokes


def test_exact_blocks_give_the_exact_inverse():
    rng = np.random.default_rng(0)
    nu_, np_ = 9, 4
    M = rng.standard_normal((nu_, nu_))
    A = M @ M.T + nu_ * np.eye(nu_)
    B = rng.standard_normal((np_, nu_))
    K = np.block([[A, B.T], [B, np.zeros((np_, np_))]])
    Ainv = np.linalg.inv(A)
    S = -B @ Ainv @ B.T
    Sinv = np.linalg.inv(S)

    class Exact(fbf.FBF):
        def __init__(self):
            self.nu_free = nu_
            self.B, self.BT = sp.csr_matrix(B), sp.csr_matrix(B.T)
            self._a = lambda r: Ainv @ r
            self._s = lambda r: Sinv @ r

    P = Exact()
    PK = np.stack([P.apply(K[:, j]) for j in range(nu_ + np_)], axis=1)
    assert np.abs(PK - np.eye(nu_ + np_)).max() < 1e-10


@pytest.mark.parametrize("k,d", [(2, 2), (3, 2), (2, 3)])
def test_star_patches_are_open_vertex_stars(k, d):
    v, c = W.unit_square_mesh(2) if d == 2 else W.kuhn_cube_mesh(1)
    V = stokes.Space(v, c, k)
    free = np.flatnonzero(~V.boundary_mask())
    patches = fbf.star_patches(V, free)
    node_to_free = -np.ones(V.n, dtype=np.int64)
    node_to_free[free] = np.arange(len(free))
    want = {}
    for ci, cell in enumerate(np.asarray(c)):
        lam = lagrange.to_barycentric(v, cell, V.coords[V.cell_nodes[ci]])
        for a, node in enumerate(V.cell_nodes[ci]):
            if node_to_free[node] < 0:
                continue
            for i, vert in enumerate(cell):
                if lam[a, i] > 1e-12:
                    want.setdefault(int(vert), set()).add(int(node_to_free[node]))
    got = {tuple(p.tolist()) for p in patches}
    assert got == {tuple(sorted(s)) for s in want.values()}


def test_pressure_mass_blocks():
    v, c = W.unit_square_mesh(2)
    v, c, _ = geometry.refine_alfeld(v, c)
    D = stokes.discretize(v, c, stokes.SV, 3)
    Mp, qn = fbf.pressure_mass_blocks(D)
    _, vol = lagrange.barycentric_gradients(D.verts, D.cells)
    assert np.allclose(Mp.sum(axis=(1, 2)), vol, rtol=1e-13)
    # global mass matrix of the SV pressure by quadrature, assembled cell by cell
    lam, w = lagrange.quadrature(2, 4)
    psi = lagrange.basis(2, 2, lam)
    Mg = np.zeros((D.Q.n, D.Q.n))
    for e in range(len(D.cells)):
        q = qn[e]
        Mg[np.ix_(q, q)] += vol[e] * np.einsum("q,qa,qb->ab", w, psi, psi)
    blk = np.zeros_like(Mg)
    for e in range(len(D.cells)):
        blk[np.ix_(qn[e], qn[e])] = Mp[e]
    assert np.abs(Mg - blk).max() < 1e-14


def test_velocity_vcycle_contracts():
    v, c = W.unit_square_mesh(2)
    vh = fbf.VelocityHierarchy(v, c, 2, [3, 2], barycentric=True)
    A = vh.levels[0].disc.K
    rng = np.random.default_rng(1)
    x_true = rng.standard_normal(A.shape[0])
    b = A @ x_true
    x = np.zeros_like(b)
    errs = []
    for _ in range(6):
        x = x + vh.vcycle(b - A @ x)
        errs.append(np.linalg.norm(x - x_true))
    rates = [errs[i + 1] / errs[i] for i in range(len(errs) - 1)]
    assert max(rates) < 0.3, rates


@pytest.mark.parametrize("k", [2, 3])
def test_fbf_fgmres_reaches_the_direct_solution(k):
    v, c = W.unit_square_mesh(2)
    rng = np.random.default_rng(2)
    meshes, _ = geometry.hierarchy(v, c, 1, True)
    nu = np.exp(0.5 * rng.standard_normal(len(meshes[0][1])))
    D = stokes.discretize(*meshes[0], stokes.SV, k, nu_cells=nu)
    sched = [k, 2] if k > 2 else [2]
    vh = fbf.VelocityHierarchy(v, c, 1, sched, barycentric=True, nu_cells=nu)
    P = fbf.FBF(D, vh, nu_cells=nu)
    f = rng.uniform(-1, 1, (2, D.V.n))
    full, its, _ = fbf.solve(P, f, tol=1e-10)
    b, xD = stokes.load_vector(D, f)
    x = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), xD))
    assert np.abs(full - x).max() < 1e-7 * np.abs(x).max()
    _, its_plain, _ = multigrid.fgmres(D.K, b, lambda r: r, tol=1e-10, maxit=2000)
    assert its < its_plain / 3, (its, its_plain)
