"""Pins of the oracle's multigrid pieces (Sec. 3, Sec. 4): Galerkin identity
of the transfers, polynomial reproduction, additive Schwarz as a dense sum,
Chebyshev closed form, Arnoldi exactness, the V-cycle as the product of the
error propagators of Eq. 3.1 / Eq. 3.2, and FGMRES' minimisation property."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import geometry, lagrange, multigrid as mg, stokes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gradual_schedule_matches_fig7():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "pmg_schedule.txt")) if l[0] != "#"]
    for k, sched in rows:
        assert mg.pmg_schedule(int(k)) == [int(s) for s in sched.split(",")]


def _pair(kind, fam=stokes.TH, kf=4, kc=2, n=2, d=2):
    v, c = W.unit_square_mesh(n) if d == 2 else W.kuhn_cube_mesh(n)
    if kind == "p":
        if fam == stokes.SV:
            v, c, _ = geometry.refine_alfeld(v, c)
        fine = stokes.discretize(v, c, fam, kf)
        coarse = stokes.discretize(v, c, stokes.TH, kc)
        f2c = np.arange(len(c))
    else:
        vf, cf, f2c = geometry.refine_uniform(v, c)
        fine = stokes.discretize(vf, cf, stokes.TH, kc)
        coarse = stokes.discretize(v, c, stokes.TH, kc)
    return fine, coarse, f2c


@pytest.mark.parametrize("case", [("p", stokes.TH, 4, 2, 2), ("p", stokes.TH, 3, 2, 3),
                                  ("p", stokes.SV, 4, 2, 2), ("h", stokes.TH, 2, 2, 2),
                                  ("h3", stokes.TH, 2, 2, 1), ("p3", stokes.TH, 3, 2, 1)])
def test_rediscretisation_equals_galerkin(case):
    """T4 (Sec. 3.1): for nested spaces and exact quadrature R K_f P = K_c."""
    kind, fam, kf, kc, n = case
    d = 3 if kind.endswith("3") else 2
    fine, coarse, f2c = _pair(kind[0], fam, kf, kc, n, d)
    P = mg.monolithic_interpolation(fine, coarse, f2c)
    G = (P.T @ fine.K @ P).toarray()
    assert np.abs(G - coarse.K.toarray()).max() < 1e-11


def test_interpolation_reproduces_polynomials():
    """T5: P I_c(q) = I_f(q) for polynomials q of the coarse degree, for the
    h-transfer (P2 on M_1 -> M_0) and the p-transfer (P2 -> P4)."""
    r = np.random.default_rng(3)
    for kind, kf, kc in [("h", 2, 2), ("p", 4, 2)]:
        fine, coarse, f2c = _pair(kind, stokes.TH, kf, kc, 2)
        PV = mg.scalar_interpolation(coarse.V, fine.V, f2c)
        a = r.normal(size=6)
        q = lambda x: a[0] + a[1] * x[:, 0] + a[2] * x[:, 1] + a[3] * x[:, 0] ** 2 + a[4] * x[:, 0] * x[:, 1] + a[5] * x[:, 1] ** 2  # noqa
        assert np.abs(PV @ q(coarse.V.coords) - q(fine.V.coords)).max() < 1e-13
        PQ = mg.scalar_interpolation(coarse.Q, fine.Q, f2c)
        ql = lambda x: a[0] + a[1] * x[:, 0] + a[2] * x[:, 1]  # noqa
        assert np.abs(PQ @ ql(coarse.Q.coords) - ql(fine.Q.coords)).max() < 1e-13


def test_vanka_patch_size_closed_form():
    """Interior TH P4/P3 patch on the structured mesh (6 cells per vertex):
    velocity nodes = 7 vertices + 12 edges * 3 + 6 cells * 3 = 61 (x2
    components), pressure = 1 + 6 edges * 2 + 6 cells * 1 = 19: n = 141.
    SV: pressure of the 6 cells, 6 * 10 = 60 (n = 182)."""
    v, c = W.unit_square_mesh(4)
    D = stokes.discretize(v, c, stokes.TH, 4)
    pt = mg.vanka_star_patches(D)
    assert max(len(p) for p in pt) == 141
    Dsv = stokes.discretize(v, c, stokes.SV, 4)
    assert max(len(p) for p in mg.vanka_star_patches(Dsv)) == 122 + 60


def test_asm_is_dense_sum_and_partition_of_unity():
    """T7 (Eq. 3.4): M^-1 e_j = sum_i I_i^T W_i K_i^-1 I_i e_j with each patch
    solve equal to numpy.linalg.solve; sum_i I_i^T W_i I_i = I."""
    v, c = W.unit_square_mesh(2)
    D = stokes.discretize(v, c, stokes.TH, 2)
    pt = mg.vanka_star_patches(D)
    asm = mg.ASM(D.K, pt)
    n = D.n_free
    Kd = D.K.toarray()
    mult = np.zeros(n)
    for p in pt:
        mult[p] += 1
    Wd = np.zeros((n, n))
    M = np.zeros((n, n))
    for p in pt:
        Ii = np.zeros((len(p), n)); Ii[np.arange(len(p)), p] = 1.0
        Wi = np.diag(1.0 / mult[p])
        M += Ii.T @ Wi @ np.linalg.solve(Ii @ Kd @ Ii.T, Ii)
        Wd += Ii.T @ Wi @ Ii
    assert np.allclose(Wd, np.eye(n), atol=1e-15)
    dense = np.stack([asm.apply(e) for e in np.eye(n)], axis=1)
    assert np.abs(dense - M).max() < 1e-11 * np.abs(M).max()


@pytest.mark.parametrize("lo,hi", [(0.1, 1.1), (0.5, 2.0)])
def test_chebyshev_matches_closed_form(lo, hi):
    """On K = diag(lam), M = I: after nu steps from x = 0 the error is
    T_nu((theta - lam)/delta) / T_nu(theta/delta) times the initial error,
    for the interval [lo, hi] * lmax."""
    lam = np.linspace(0.05, 2.0, 40)
    K = sp.diags(lam).tocsr()
    xs = np.random.default_rng(0).normal(size=40)
    b = K @ xs
    lmax = 2.0
    for nu in (1, 2, 3, 5):
        x = mg.chebyshev(K, lambda r: r, b, np.zeros(40), nu, lmax, lo, hi)
        a, bb = lo * lmax, hi * lmax
        th, de = (a + bb) / 2, (bb - a) / 2
        tt = (th - lam) / de
        inside = np.abs(tt) <= 1
        Tn = np.cos(nu * np.arccos(np.clip(tt, -1, 1)))
        out = np.cosh(nu * np.arccosh(np.maximum(np.abs(tt), 1.0))) * np.sign(tt) ** nu
        Tn = np.where(inside, Tn, out)
        want = Tn / np.cosh(nu * np.arccosh(th / de)) * xs
        assert np.abs((xs - x) - want).max() < 1e-12


def test_arnoldi_exact_on_small_operators():
    """10 Arnoldi steps span the whole space of a 6x6 operator: the estimate
    equals the largest real part of its exact eigenvalues."""
    r = np.random.default_rng(2)
    A = r.normal(size=(6, 6)) + 4 * np.eye(6)
    K = sp.csr_matrix(A)
    est = mg.arnoldi_lmax(K, lambda x: x, r.normal(size=6), 10)
    assert abs(est - np.linalg.eigvals(A).real.max()) < 1e-10
    Minv = np.diag(1 / np.arange(1, 7.0))
    est = mg.arnoldi_lmax(K, lambda x: Minv @ x, r.normal(size=6), 10)
    assert abs(est - np.linalg.eigvals(Minv @ A).real.max()) < 1e-10


def _dense(op, n):
    return np.stack([op(e) for e in np.eye(n)], axis=1)


def test_vcycle_equals_error_propagator_products():
    """T6: with r = K x the V-cycle's error propagator I - B K equals the
    product of Eq. 3.1 (hMG) and Eq. 3.2 (phMG defect correction), with
    nu = 1 Chebyshev = damped ASM (I - w M^-1 K) and the exact coarse solve."""
    v, c = W.unit_square_mesh(2)   # a 1x1 coarsest mesh has spurious pressure modes
    h = mg.Hierarchy(v, c, 1, stokes.TH, [3, 2], opts=mg.Options(n_V=2))
    L0, L1, L2 = h.levels
    assert [L.kind for L in h.levels] == ["p", "h", "coarse"]
    n0, n1, n2 = (L.disc.n_free for L in h.levels)
    K0, K1 = L0.disc.K.toarray(), L1.disc.K.toarray()
    C = _dense(h.coarse_solve, n2)
    def S(L, n):
        w = 2.0 / (1.2 * L.lmax)
        return np.eye(n) - w * _dense(L.asm.apply, n) @ L.disc.K.toarray()
    T1 = 2.0 / (1.2 * L1.lmax) * _dense(L1.asm.apply, n1)
    P1, R1 = L1.P.toarray(), L1.R.toarray()
    # hMG two-grid operator on level 1 (Eq. 3.1) written as B_1
    B1 = T1 + (np.eye(n1) - T1 @ K1) @ (T1 + P1 @ C @ R1 @ (np.eye(n1) - K1 @ T1))
    assert np.abs(_dense(lambda r: h.hcycle(1, r), n1) - B1).max() < 1e-10 * np.abs(B1).max()
    # n_V = 2 hMG cycles: B = B1 + B1 (I - K1 B1)
    Bn = B1 + B1 @ (np.eye(n1) - K1 @ B1)
    P0, R0 = L0.P.toarray(), L0.R.toarray()
    S0 = S(L0, n0)
    G0 = S0 @ (np.eye(n0) - P0 @ Bn @ R0 @ K0) @ S0          # Eq. 3.2
    B0 = _dense(h.vcycle, n0)
    assert np.abs((np.eye(n0) - B0 @ K0) - G0).max() < 1e-9


def test_fgmres_properties():
    """FGMRES: with the exact inverse as preconditioner it stops after one
    iteration; with the V-cycle it converges to the sparse direct solution
    within tol * cond; the k-th iterate minimises ||b - K x|| over span(Z_k)."""
    v, c = W.unit_square_mesh(2)
    h = mg.Hierarchy(v, c, 1, stokes.TH, [2])
    D = h.levels[0].disc
    f = W.nodal_forcing(D.V.n, 2, 1)
    b, xD = stokes.load_vector(D, f)
    x_ref = stokes.direct_solve(D, b)
    x, its, hist = mg.fgmres(D.K, b, lambda r: stokes.direct_solve(D, r), tol=1e-10)
    assert its == 1
    x, its, hist = mg.fgmres(D.K, b, h.vcycle, tol=1e-12)
    pm = D.pressure_mask_free()
    dx = x - x_ref
    dx[pm] -= dx[pm].mean()
    assert np.linalg.norm(dx) < 1e-8 * np.linalg.norm(x_ref)
    assert np.all(np.diff(hist) <= 1e-15)          # monotone residual
    # minimisation property after 3 iterations
    x3, its3, h3 = mg.fgmres(D.K, b, h.vcycle, tol=1e-30, maxit=3)
    Z = np.stack([v for v in _krylov_Z(D.K, b, h.vcycle, 3)], axis=1)
    y, *_ = np.linalg.lstsq(D.K @ Z, b, rcond=None)
    assert abs(np.linalg.norm(b - D.K @ x3) - np.linalg.norm(b - D.K @ Z @ y)) < 1e-10 * np.linalg.norm(b)


def _krylov_Z(K, b, M, m):
    """Z_k of flexible GMRES rebuilt independently with classical
    Gram-Schmidt applied twice."""
    V = [b / np.linalg.norm(b)]
    Z = []
    for j in range(m):
        z = M(V[j]); Z.append(z)
        w = K @ z
        for _ in range(2):
            for vv in V:
                w = w - (w @ vv) * vv
        V.append(w / np.linalg.norm(w))
    return Z


@pytest.mark.slow
def test_phmg_solver_converges_and_matches_direct():
    """The full FGMRES-phMG solve on the manufactured TH P2 8x8 problem
    reaches 1e-10 and agrees with the sparse direct solution; the errors
    against the exact solution are the discretisation errors."""
    w = W.workload("th_p2_8x8")
    h = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule)
    D = h.levels[0].disc
    f = W.mms_forcing(D.V.coords).T
    g = W.mms_velocity(D.V.coords).T
    full, its, hist, b, x = mg.solve(h, f, g, tol=1e-12)
    assert its < 40
    xd = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), stokes.load_vector(D, f, g)[1]))
    assert np.abs(full - xd).max() < 1e-9


@pytest.mark.parametrize("mesh", [("square", 2), ("square", 4), ("cube", 2)])
def test_bordered_coarse_solve_is_the_zero_mean_solution(mesh):
    """The coarsest solve (Sec. 4: exact; Sec. 2: p in L^2_0) returns, for a
    consistent right-hand side r (pressure part orthogonal to the constant
    null vector n of K), the unique x with K x = r and int p_h = 0.  Pinned
    without the oracle's LU: the minimum-norm least-squares solution of the
    dense K (SVD) moved along n until int p_h = 0, with the pressure
    integrals summing to the domain's measure."""
    kind, n = mesh
    v, c = W.unit_square_mesh(n) if kind == "square" else W.kuhn_cube_mesh(n)
    h = mg.Hierarchy(v, c, 1, stokes.TH, [2])
    D = h.levels[-1].disc
    assert len(D.cells) == len(c)                       # the coarsest level is the input mesh
    nf = D.n_free
    pm = D.pressure_mask_free()
    w = D.p_integrals[D.free[pm] - D.d * D.V.n]         # int psi_j of the free pressures
    assert abs(w.sum() - 1.0) < 1e-12                   # |unit square| = |unit cube| = 1
    nullv = np.zeros(nf)
    nullv[pm] = 1.0
    K = D.K.toarray()
    assert np.abs(K @ nullv).max() < 1e-12 * np.abs(K).max()
    r = np.random.default_rng(n).standard_normal(nf)
    r[pm] -= r[pm].mean()                               # consistent: n . r = 0
    x = h.coarse_solve(r)
    assert np.abs(K @ x - r).max() < 1e-11 * np.abs(r).max()
    assert abs(w @ x[pm]) < 1e-13 * np.abs(x).max()
    y = np.linalg.lstsq(K, r, rcond=1e-12)[0]           # orthogonal to n
    ref = y - (w @ y[pm]) / w.sum() * nullv
    assert np.abs(x - ref).max() < 1e-10 * np.abs(ref).max()
    # the constant null space is the only one (the border makes K uniquely solvable)
    s = np.linalg.svd(K, compute_uv=False)
    assert s[-1] < 1e-12 * s[0] < s[-2]


def test_tight_fgmres_reaches_the_discrete_solution():
    """FGMRES-phMG run to a relative residual of 1e-14 (with the V(2,2)
    relaxation on [0.5, 2.0] lambda_hat) gives the discrete solution of
    Eq. 2.3 on the 16x16 P4/P3 problem: u and the zero-mean p agree with the
    bordered sparse LU solve (with one refinement step) to 1e-11, relative to
    their max norms.  The GPU parity test of the full-size P4/P3 problem
    compares with this tight oracle solve."""
    v, c = W.unit_square_mesh(8)
    h = mg.Hierarchy(v, c, 1, stokes.TH, [4, 2],
                     opts=mg.Options(nu_p=2, nu_h=2, cheb_lo=0.5, cheb_hi=2.0, eig_steps=8))
    D = h.levels[0].disc
    f = W.nodal_forcing(D.V.n, D.d, 0)
    full, its, hist, b, x = mg.solve(h, f, None, tol=1e-14)
    assert hist[-1] <= 1e-14 and its < 30
    xd = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), np.zeros(D.n_full)))
    nu = D.d * D.V.n
    assert np.abs(full[:nu] - xd[:nu]).max() < 1e-11 * np.abs(xd[:nu]).max()
    assert np.abs(full[nu:] - xd[nu:]).max() < 1e-11 * np.abs(xd[nu:]).max()
