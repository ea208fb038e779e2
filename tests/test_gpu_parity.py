"""GPU parity of every hot-path step against the FP64 oracle, through the C
ABI (small meshes that still span many patches, ragged boundary patches and
several levels).

Tolerances (relative to the max-norm of the oracle's result):
  FP64 steps    1e-11 (SpMV, transfers: a few ulp times the row length),
                1e-10 (patch inverses, ASM, V-cycle: Gauss-Jordan vs LAPACK
                LU differ by cond(K_i) * eps, cond(K_i) <= 1e4 here),
  FP32 steps    2e-5 (SpMV / transfers, 4 eps32 * row sum / max),
                2e-4 (ASM and V-cycle with FP32 inverses: eps32 * cond(K_i)),
  FGMRES        relative residual <= tol on both sides; solved to 1e-13,
                velocity and zero-mean pressure within 1e-10 relative
                (tol * cond(K), cond(K) <= 1e3 on these meshes).
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg, rng, stokes
from tests.dofmap import full_field_perms, keys, level_perm, permutation

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

CASES = {
    "th_p2_8x8": (W.unit_square_mesh(2), 2, 0, 2, [2], False),
    "th_p4_8x8": (W.unit_square_mesh(2), 2, 0, 4, [4, 2], False),
    "th_p4_gradual": (W.unit_square_mesh(2), 2, 0, 4, [4, 3, 2], False),
    "sv_p3_alfeld": (W.unit_square_mesh(2), 2, 1, 3, [3, 2], True),
    "sv_p4_disk": (W.delaunay_disk_mesh(0, h=0.4), 1, 1, 4, [4, 2], True),
    "th3d_p3": (W.kuhn_cube_mesh(2), 1, 0, 3, [3, 2], False),
}

_cache = {}


def dev():
    return torch.device("cuda:0")


def pair(name, precision=P.FP64, **o):
    key = (name, precision, tuple(sorted(o.items())))
    if key in _cache:
        return _cache[key]
    (v, c), nref, fam, k, sched, bary = CASES[name]
    opts = mg.Options(nu_p=o.get("nu_p", 1), nu_h=o.get("nu_h", 1), n_V=o.get("n_V", 1),
                      cheb_lo=o.get("cheb_lo", 0.1), cheb_hi=o.get("cheb_hi", 1.1))
    # the oracle has one exact patch solve; patch_solver only selects the library's kernel
    ora = mg.Hierarchy(v, c, nref, fam, sched, barycentric=bary, opts=opts)
    lm = [L.lmax for L in ora.levels[:-1]]
    h = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched,
                   lmax_override=lm, precision=precision, **o)
    perms = [level_perm(h, li, L.disc) for li, L in enumerate(ora.levels)]
    _cache[key] = (h, ora, perms)
    return _cache[key]


def to_lib(x_o, perm):
    x = np.empty_like(x_o)
    x[perm] = x_o
    return torch.tensor(x, device=dev())


def from_lib(t, perm):
    return t.cpu().numpy()[perm]


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


NAMES = list(CASES)


@pytest.mark.parametrize("name", NAMES)
def test_a1_patch_gather_is_exact(name):
    """a1: the device gather equals the library's own CSR entries bit for bit
    and the oracle's patch blocks to rounding."""
    h, ora, perms = pair(name)
    for li, L in enumerate(ora.levels[:-1]):
        got = h.patch_matrices(li)
        off, dofs = h.patches(li)
        K = h.get_csr(li, 0).tocsr()
        pos = 0
        inv = np.argsort(perms[li])
        ora_blocks = {tuple(p.tolist()): b for p, b in zip(L.asm.patches, L.asm.blocks)}
        for i in range(len(off) - 1):
            d = dofs[off[i]:off[i + 1]]
            n = len(d)
            blk = got[pos:pos + n * n].reshape(n, n)
            pos += n * n
            assert np.array_equal(blk, K[d][:, d].toarray())
            od = inv[d]
            order = np.argsort(od)
            ob = ora_blocks[tuple(od[order].tolist())]
            assert np.abs(blk[np.ix_(order, order)] - ob).max() <= 1e-12 * np.abs(ob).max()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("solver", [0, 1])
def test_a2_patch_inverses(name, solver):
    """a2: the batched FP64 patch inverses (0: saddle block inverse, 1:
    partial-pivot Gauss-Jordan) equal the inverse of the oracle's patch block
    (LAPACK LU) to cond * eps."""
    h, ora, perms = pair(name, patch_solver=solver)
    for li, L in enumerate(ora.levels[:-1]):
        got = h.patch_inverses(li)
        off, dofs = h.patches(li)
        inv = np.argsort(perms[li])
        ora_blocks = {tuple(p.tolist()): b for p, b in zip(L.asm.patches, L.asm.blocks)}
        pos = 0
        for i in range(len(off) - 1):
            d = dofs[off[i]:off[i + 1]]
            n = len(d)
            Ki = got[pos:pos + n * n].reshape(n, n)
            pos += n * n
            od = inv[d]
            order = np.argsort(od)
            ob = ora_blocks[tuple(od[order].tolist())]
            ref = np.linalg.inv(ob)
            assert relerr(Ki[np.ix_(order, order)], ref) < 1e-10


@pytest.mark.parametrize("name", ["th_p2_8x8", "th_p4_8x8", "sv_p3_alfeld", "th3d_p3"])
def test_a3_arnoldi_lambda_max(name):
    """a3: the device Arnoldi estimate equals the oracle's from the same start
    vector; the default setup draws its SplitMix64 start vector by library
    DoF index, which the oracle reproduces through the permutation."""
    h, ora, perms = pair(name)
    for li, L in enumerate(ora.levels[:-1]):
        v0 = np.random.default_rng(li).standard_normal(L.disc.n_free)
        got = h.arnoldi_lmax(li, to_lib(v0, perms[li]), 10)
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, 10)
        assert abs(got - want) <= 1e-9 * abs(want)
    (v, c), nref, fam, k, sched, bary = CASES[name]
    hd = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched)
    lm = hd.info()["lmax"]
    for li, L in enumerate(ora.levels[:-1]):
        v0 = rng.uniform_pm1(0, li, perms[li])
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, mg.Options().eig_steps)
        assert abs(lm[li] - want) <= 1e-9 * abs(want)
    hd.close()
    # mixed precision: the same Arnoldi with M^{-1} K applied in FP32 (FP32 CSR
    # values and stored inverses); the basis stays FP64
    hm = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched,
                    precision=P.MIXED)
    lmm = hm.info()["lmax"]
    for li, L in enumerate(ora.levels[:-1]):
        v0 = rng.uniform_pm1(0, li, perms[li])
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, mg.Options().eig_steps)
        assert abs(lmm[li] - want) <= 1e-4 * abs(want), (li, lmm[li], want)
    hm.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_a4_a6_residual_and_transfers(name, precision):
    """a4 r = b - K x and a6 restriction / prolongation on every level."""
    h, ora, perms = pair(name, precision)
    tol = 1e-11 if precision == P.FP64 else 2e-5
    g = np.random.default_rng(7)
    for li, L in enumerate(ora.levels):
        n = L.disc.n_free
        b, x = g.standard_normal(n), g.standard_normal(n)
        r = from_lib(h.residual(li, to_lib(b, perms[li]), to_lib(x, perms[li]), precision), perms[li])
        want = b - L.disc.K @ x
        scale = np.abs(b).max() + np.abs(L.disc.K).max() * np.abs(x).max() * 10
        assert np.abs(r - want).max() <= tol * scale
        if li + 1 < len(ora.levels):
            xf = g.standard_normal(n)
            yc = torch.zeros(ora.levels[li + 1].disc.n_free, dtype=torch.float64, device=dev())
            h.transfer(li, 0, to_lib(xf, perms[li]), yc, precision)
            assert relerr(from_lib(yc, perms[li + 1]), L.R @ xf) <= tol * 10
            xc = g.standard_normal(ora.levels[li + 1].disc.n_free)
            y0 = g.standard_normal(n)
            yf = to_lib(y0, perms[li])
            h.transfer(li, 1, to_lib(xc, perms[li + 1]), yf, precision)
            assert relerr(from_lib(yf, perms[li]), y0 + L.P @ xc) <= tol * 10


@pytest.mark.parametrize("name", NAMES)
def test_a6_device_transfers_equal_host_transfers(name):
    """a6: P and R = P^T built on the device (the GPU setup) equal the host
    construction of the same library (host_only handle) entry by entry:
    identical sparsity with sorted rows, values to rounding (the device
    evaluates the coarse basis at the fine nodes from the mesh geometry or
    from a lattice table; the host from its own tables)."""
    h, ora, perms = pair(name)
    (v, c), nref, fam, k, sched, bary = CASES[name]
    hh = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, host_only=1)
    for li in range(len(ora.levels) - 1):
        for which in (1, 2):
            A, B = h.get_csr(li, which), hh.get_csr(li, which)
            assert A.shape == B.shape
            assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices), (li, which)
            assert np.abs(A.data - B.data).max() <= 1e-13 * np.abs(B.data).max(), (li, which)
    hh.close()


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_a5_additive_schwarz(name, precision):
    """a5: z = sum_i I_i^T W_i K_i^{-1} I_i r (Eq. 3.4)."""
    h, ora, perms = pair(name, precision)
    tol = 1e-10 if precision == P.FP64 else 2e-4
    for li, L in enumerate(ora.levels[:-1]):
        r = np.random.default_rng(li).standard_normal(L.disc.n_free)
        z = from_lib(h.asm(li, to_lib(r, perms[li]), precision), perms[li])
        assert relerr(z, L.asm.apply(r)) < tol


@pytest.mark.parametrize("name", NAMES)
def test_a7_coarse_solve(name):
    """a7: bordered FP64 LU solve of the coarsest level."""
    h, ora, perms = pair(name)
    L = ora.levels[-1]
    r = np.random.default_rng(3).standard_normal(L.disc.n_free)
    pm = L.disc.pressure_mask_free()
    r[pm] -= r[pm].mean()
    x = from_lib(h.coarse_solve(to_lib(r, perms[-1])), perms[-1])
    assert relerr(x, ora.coarse_solve(r)) < 1e-10


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_vcycle_matches_oracle(name, precision):
    """The whole phMG V-cycle (Eq. 3.2 / 3.1 with the exact coarse solve)."""
    h, ora, perms = pair(name, precision)
    r = np.random.default_rng(11).standard_normal(ora.levels[0].disc.n_free)
    z = from_lib(h.vcycle(to_lib(r, perms[0])), perms[0])
    assert relerr(z, ora.vcycle(r)) < (1e-10 if precision == P.FP64 else 2e-4)


@pytest.mark.parametrize("o", [dict(nu_p=2, nu_h=2), dict(nu_p=3, nu_h=1, n_V=2), dict(n_V=2),
                               dict(nu_p=2, nu_h=2, cheb_lo=0.5, cheb_hi=2.0)])
def test_vcycle_chebyshev_degrees_and_nV(o):
    """Chebyshev degree > 1 and n_V > 1 (the (n_V, nu_p, nu_h) family of
    Sec. 4.1.1), and another Chebyshev interval, in both precisions."""
    for precision in (P.FP64, P.MIXED):
        h, ora, perms = pair("th_p4_8x8", precision, **o)
        r = np.random.default_rng(5).standard_normal(ora.levels[0].disc.n_free)
        z = from_lib(h.vcycle(to_lib(r, perms[0])), perms[0])
        assert relerr(z, ora.vcycle(r)) < (1e-10 if precision == P.FP64 else 5e-4)


def test_vcycle_many_rhs_and_determinism():
    """nrhs > 1 runs each right-hand side; repeated runs are bitwise equal
    (no atomics in the scatter)."""
    h, ora, perms = pair("th_p4_8x8")
    n = ora.levels[0].disc.n_free
    R = torch.randn(3, n, dtype=torch.float64, device=dev())
    Z1 = h.vcycle(R)
    Z2 = h.vcycle(R)
    assert torch.equal(Z1, Z2)
    for q in range(3):
        assert torch.equal(h.vcycle(R[q].clone()), Z1[q])


def _solve_pair(name, precision, tol, tol_oracle=None):
    h, ora, perms = pair(name, precision)
    D = ora.levels[0].disc
    pv, pq = full_field_perms(h, D)
    g = np.random.default_rng(2)
    f_o = g.uniform(-1, 1, size=(D.d, D.V.n))
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    u, p, its, rel = h.solve(torch.tensor(f_l.reshape(-1), device=dev()), tol=tol)
    full, its_o, hist, b, x = mg.solve(ora, f_o, None, tol=tol if tol_oracle is None else tol_oracle)
    U = u.cpu().numpy().reshape(D.d, -1)[:, pv]
    Pp = p.cpu().numpy()[pq]
    nV = D.V.n
    uo = full[:D.d * nV].reshape(D.d, nV)
    po = full[D.d * nV:]
    return U, Pp, its, rel, uo, po, its_o, D


@pytest.mark.parametrize("name", ["th_p2_8x8", "th_p4_8x8", "sv_p3_alfeld", "th3d_p3"])
def test_fgmres_solve_fp64(name):
    """a8: FGMRES-phMG in FP64 reaches the tolerance in the oracle's number
    of iterations (+-1), and its solution (velocity and zero-mean pressure,
    Sec. 2: p in L^2_0) equals the oracle's to 1e-10 relative in the max norm
    when both solve to 1e-13 (error <= cond(K) * tol, cond(K) <= 1e3 here)."""
    U, Pp, its, rel, uo, po, its_o, D = _solve_pair(name, P.FP64, 1e-13)
    assert rel <= 1e-13 and abs(its - its_o) <= 1, (its, its_o)
    assert relerr(U, uo) < 1e-10
    assert relerr(Pp, po) < 1e-10
    assert abs(D.p_integrals @ Pp) < 1e-12 * np.abs(Pp).max()


@pytest.mark.parametrize("name", ["th_p4_8x8", "sv_p3_alfeld", "th3d_p3"])
def test_fgmres_solve_mixed(name):
    """Mixed precision (FP32 V-cycle inside FP64 FGMRES): the FP32
    preconditioner only changes the Krylov space, so the flexible FP64
    iteration still reaches 1e-13 and the FP64 solution to 1e-10, in at most
    a few more iterations than the oracle."""
    U, Pp, its, rel, uo, po, its_o, D = _solve_pair(name, P.MIXED, 1e-13)
    assert rel <= 1e-13 and its <= its_o + 5, (its, its_o)
    assert relerr(U, uo) < 1e-10
    assert relerr(Pp, po) < 1e-10


def test_manufactured_solution_with_lifting_and_viscosity():
    """Dirichlet lifting, constant nu scaling and the zero-mean pressure."""
    h, ora, perms = pair("th_p2_8x8")
    D = ora.levels[0].disc
    vx, px, _ = h.nodes()
    pv = permutation(keys(vx, np.zeros(len(vx))), keys(D.V.coords, np.zeros(D.V.n)))
    pq = permutation(keys(px, np.zeros(len(px))), keys(D.Q.coords, np.zeros(D.Q.n)))
    nu = 2.5
    f = torch.tensor((nu * W.mms_forcing(vx)).T.copy().reshape(-1), device=dev())
    g = torch.tensor(W.mms_velocity(vx).T.copy().reshape(-1), device=dev())
    u, p, its, rel = h.solve(f, g, nu=nu, tol=1e-12)
    # oracle with nu: scale f, then p_h -> nu * p'
    full, _, _, _, _ = mg.solve(ora, W.mms_forcing(D.V.coords).T, W.mms_velocity(D.V.coords).T, tol=1e-12)
    nV = D.V.n
    U = u.cpu().numpy().reshape(2, -1)[:, pv]
    Pp = p.cpu().numpy()[pq]
    assert relerr(U, full[:2 * nV].reshape(2, nV)) < 1e-9
    assert relerr(Pp, nu * full[2 * nV:]) < 1e-8     # p scales with nu
    assert abs(D.p_integrals @ Pp) < 1e-12


def test_error_paths_are_reported():
    """Failures come back as status codes, never as device faults: NaN in f
    (ENONFINITE), maxit reached (ENOTCONVERGED), a zero pivot in every patch
    (nu = 0 makes the velocity block vanish: ESINGULAR), zero RHS (0 its)."""
    (v, c), nref, fam, k, sched, bary = CASES["th_p2_8x8"]
    h = P.StokesMG(v, c, nref, fam, k, maxit=2)
    nV = h.info()["n_vel_nodes"]
    f = torch.zeros(2 * nV, dtype=torch.float64, device=dev())
    u, p, its, rel = h.solve(f)
    assert its == 0 and float(u.abs().max()) == 0.0
    f.uniform_(-1, 1)
    with pytest.raises(P.StokesError) as e:
        h.solve(f, tol=1e-12)
    assert e.value.code == -4
    f[5] = float("nan")
    with pytest.raises(P.StokesError) as e:
        h.solve(f)
    assert e.value.code == -5
    h.close()
    with pytest.raises(P.StokesError) as e:
        P.StokesMG(v, c, nref, fam, k, nu_cell=np.zeros(128))
    assert e.value.code == -3
