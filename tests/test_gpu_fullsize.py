"""Parity at the workloads' full sizes, in the launch configuration that
bench.py times (HIER_EXPLICIT schedule, bench's relaxation parameters,
defaults otherwise).

* TH P4/P3 on the 64x64 square (167,299 free DoFs, the benchmark workload),
  with both relaxations bench times (Chebyshev degree 2 on [0.5, 2.0]
  lambda_max from 8 Arnoldi steps, and degree 1 on [0.1, 1.1] lambda_max
  from 15): lambda_max of every
  level from the library's SplitMix64 start vector (FP64 handle 1e-9; the
  mixed handle's FP32 operator within 1e-4), one V-cycle in FP64 (1e-10) and
  in mixed precision (2e-4) against the oracle's V-cycle with the same
  lambda_max, FGMRES iteration counts (+-1).
* The same workload solved to 1e-13 in FP64 and in mixed precision: velocity
  and zero-mean pressure equal the oracle's tight solution to 1e-10.
* SV P4/P3disc on the Alfeld-refined Delaunay disk and TH P3/P2 on the 16^3
  Kuhn cube: the library's solution, mapped to the oracle's DoFs, has a true
  relative residual <= 2e-8 under the oracle's independently assembled
  operator and load (the solver stops at 1e-8 on its own operator; the two
  operators differ by rounding), and sampled patch inverses match
  numpy.linalg.inv of the oracle's blocks.
* FBF(phMG) on the SV disk: the same true-residual check.
* The batched V-cycle on the 16^3 cube with 64 right-hand sides: every column
  against the single-vector mixed V-cycle.
* The viscosity gradient on 128^2 with per-cell viscosity: a directional
  central difference of the library's own solves.
* The bench's relaxation keeps the FGMRES iteration count flat from 64^2 to
  128^2 (a property of the method under these parameters, not a parity check).
* The bench's 32-forcing batched forward and adjoint on 128^2 with per-cell
  viscosity: sampled columns' true residuals under the oracle's operator, and
  the batched viscosity gradient against the per-column sum.
"""
import numpy as np
import pytest

import workloads as W
from oracle import geometry, multigrid as mg, rng, stokes
from tests.dofmap import full_field_perms, keys, level_perm, permutation

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _lib(w, precision, **o):
    return P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric,
                      hierarchy=P.HIER_EXPLICIT, schedule=w.schedule, precision=precision, **o)


def _to_lib(x_o, perm):
    x = np.empty_like(x_o)
    x[perm] = x_o
    return torch.tensor(x, device="cuda")


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


_ORA64 = {}


@pytest.mark.parametrize("relax", ["v22", "v11"])
def test_benchmark_workload_th_p4_64x64(relax):
    from bench import RELAX
    o = RELAX[relax]
    w = W.workload("th_p4_64x64")
    if "ora" not in _ORA64:
        _ORA64["ora"] = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule, lmax=[1.0] * 16)
    ora = _ORA64["ora"]
    ora.opts = mg.Options(**o)           # the relaxation only enters the cycle, not the setup
    h64 = _lib(w, P.FP64, **o)
    hmx = _lib(w, P.MIXED, **o)
    perms = [level_perm(h64, li, L.disc) for li, L in enumerate(ora.levels)]
    lm = h64.info()["lmax"]
    # mixed mode applies M^{-1} K in FP32 inside the FP64-orthogonalised Arnoldi
    for a, b in zip(hmx.info()["lmax"][:len(lm) - 1], lm[:len(lm) - 1]):
        assert abs(a - b) <= 1e-4 * b, (a, b)
    for li, L in enumerate(ora.levels[:-1]):
        v0 = rng.uniform_pm1(0, li, perms[li])
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, ora.opts.eig_steps)
        assert abs(lm[li] - want) <= 1e-9 * want, (li, lm[li], want)
        L.lmax = lm[li]
    r = np.random.default_rng(1).standard_normal(ora.levels[0].disc.n_free)
    z_o = ora.vcycle(r)
    z64 = h64.vcycle(_to_lib(r, perms[0])).cpu().numpy()[perms[0]]
    zmx = hmx.vcycle(_to_lib(r, perms[0])).cpu().numpy()[perms[0]]
    assert _relerr(z64, z_o) < 1e-10
    assert _relerr(zmx, z_o) < 2e-4
    # FGMRES to 1e-8 with the same lambda_max: iteration counts agree
    D = ora.levels[0].disc
    vx, _, _ = h64.nodes()
    pv = permutation(keys(vx, np.zeros(len(vx))), keys(D.V.coords, np.zeros(D.V.n)))
    f_o = W.nodal_forcing(D.V.n, 2, 0)
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    f_t = torch.tensor(f_l.reshape(-1), device="cuda")
    _, _, its64, rel64 = h64.solve(f_t, tol=1e-8)
    _, _, itsmx, relmx = hmx.solve(f_t, tol=1e-8)
    _, its_o, _, _, _ = mg.solve(ora, f_o, None, tol=1e-8)
    assert rel64 <= 1e-8 and relmx <= 1e-8
    assert abs(its64 - its_o) <= 1, (its64, its_o)
    assert itsmx <= its_o + 3, (itsmx, its_o)
    h64.close()
    hmx.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solution_matches_oracle_to_1e10_at_bench_size(precision):
    """The FP64 accuracy target on the benchmark workload (TH P4/P3 on the
    64x64 square, 167,299 free DoFs, the bench's V(2,2) relaxation): the
    library's FGMRES-phMG solved to a relative residual of 1e-13 gives the
    oracle's solution (FGMRES-phMG to 1e-14, which equals the refined sparse
    direct solve on the 16x16 problem to 1e-11) to 1e-10 relative in the
    max norm, for the velocity and for the zero-mean pressure (Sec. 2:
    p in L^2_0).  The mixed path (FP32 V-cycle inside FP64 FGMRES) reaches
    the same solution: its preconditioner's rounding only shapes the Krylov
    space."""
    from bench import RELAX
    o = RELAX["v22"]
    w = W.workload("th_p4_64x64")
    if "ora" not in _ORA64:
        _ORA64["ora"] = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule, lmax=[1.0] * 16)
    ora = _ORA64["ora"]
    ora.opts = mg.Options(**o)
    h = _lib(w, P.FP64 if precision == "fp64" else P.MIXED, **o)
    for L, lm in zip(ora.levels[:-1], h.info()["lmax"]):
        L.lmax = lm
    D = ora.levels[0].disc
    pv, pq = full_field_perms(h, D)
    f_o = W.nodal_forcing(D.V.n, 2, 0)
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    u, p, its, rel = h.solve(torch.tensor(f_l.reshape(-1), device="cuda"), tol=1e-13)
    assert rel <= 1e-13
    if "full" not in _ORA64:
        _ORA64["full"] = mg.solve(ora, f_o, None, tol=1e-14)[0]
    full = _ORA64["full"]
    nV = D.V.n
    U = u.cpu().numpy().reshape(2, -1)[:, pv]
    Pp = p.cpu().numpy()[pq]
    eu = _relerr(U, full[:2 * nV].reshape(2, nV))
    ep = _relerr(Pp, full[2 * nV:])
    assert eu < 1e-10 and ep < 1e-10, (eu, ep, its)
    assert abs(D.p_integrals @ Pp) < 1e-12 * np.abs(Pp).max()
    h.close()


def _true_residual_case(name, n_sample=24):
    w = W.workload(name)
    meshes, _ = geometry.hierarchy(w.verts, w.cells, w.n_refine, w.barycentric)
    D = stokes.discretize(*meshes[0], w.family, w.k)
    h = _lib(w, P.MIXED)
    perm = level_perm(h, 0, D)
    vx, _, _ = h.nodes()
    pv = permutation(keys(vx, np.zeros(len(vx))), keys(D.V.coords, np.zeros(D.V.n)))
    f_o = W.nodal_forcing(D.V.n, D.d, w.seed)
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    u, p, its, rel = h.solve(torch.tensor(f_l.reshape(-1), device="cuda"), tol=1e-8)
    assert rel <= 1e-8
    b, xD = stokes.load_vector(D, f_o)
    pv2, pq = full_field_perms(h, D)
    U = u.cpu().numpy().reshape(D.d, -1)[:, pv2].reshape(-1)
    x_full = np.concatenate([U, p.cpu().numpy()[pq]])
    x = x_full[D.free]
    res = np.linalg.norm(b - D.K @ x) / np.linalg.norm(b)
    assert res <= 2e-8, res
    # sampled patch inverses against numpy on the oracle's blocks
    off, dofs = h.patches(0)
    invs = h.patch_inverses(0)
    start = np.concatenate([[0], np.cumsum(np.diff(off).astype(np.int64) ** 2)])
    inv_perm = np.argsort(perm)
    sel = np.random.default_rng(3).choice(len(off) - 1, size=min(n_sample, len(off) - 1), replace=False)
    Kc = D.K.tocsr()
    for i in sel:
        dl = dofs[off[i]:off[i + 1]]
        n = len(dl)
        od = inv_perm[dl]
        blk = Kc[od][:, od].toarray()
        got = invs[start[i]:start[i] + n * n].reshape(n, n)
        assert _relerr(got, np.linalg.inv(blk)) < 1e-9
    h.close()
    return its


def test_scott_vogelius_disk_true_residual():
    _true_residual_case("sv_p4_disk")


def test_taylor_hood_3d_cube_true_residual():
    _true_residual_case("th_p3_cube16", n_sample=12)


def test_fbf_disk_true_residual():
    """FBF(phMG) (Eq. fbf) on the SV P4 disk at full size: the solution's true
    residual under the oracle's independently assembled operator <= 2e-8, and
    the solve stays within the monolithic solver's iteration range (the paper
    reports FBF(phMG) as robust for SV)."""
    w = W.workload("sv_p4_disk")
    meshes, _ = geometry.hierarchy(w.verts, w.cells, w.n_refine, w.barycentric)
    D = stokes.discretize(*meshes[0], w.family, w.k)
    h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, fbf=True, hierarchy=P.HIER_EXPLICIT,
                   schedule=w.schedule, precision=P.MIXED)
    pv, pq = full_field_perms(h, D)
    f_o = W.nodal_forcing(D.V.n, D.d, w.seed)
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    u, p, its, rel = h.solve(torch.tensor(f_l.reshape(-1), device="cuda"), tol=1e-8)
    assert rel <= 1e-8 and its <= 40, (rel, its)
    b, _ = stokes.load_vector(D, f_o)
    U = u.cpu().numpy().reshape(D.d, -1)[:, pv].reshape(-1)
    x = np.concatenate([U, p.cpu().numpy()[pq]])[D.free]
    res = np.linalg.norm(b - D.K @ x) / np.linalg.norm(b)
    assert res <= 2e-8, res
    h.close()


def test_batched_columns_match_single_vcycle_on_cube16():
    """The batched V-cycle in bench's configuration (TH P3/P2 on the 16^3
    cube, 64 right-hand sides): every column of the 3xTF32 batch equals the
    single-vector mixed V-cycle to 1e-4 and every TF32 column to 2e-2 (the
    accuracy argument of tests/test_gpu_batched.py holds at any size)."""
    w = W.workload("th_p3_cube16")
    h = _lib(w, P.MIXED)
    n = h.info()["n_free"][0]
    R = torch.tensor(np.random.default_rng(4).standard_normal((64, n)), device="cuda")
    Z1 = h.vcycle(R)
    scale = Z1.abs().amax(dim=1)
    e3 = ((h.vcycle_batched(R, P.BATCH_3XTF32) - Z1).abs().amax(dim=1) / scale).max().item()
    et = ((h.vcycle_batched(R, P.BATCH_TF32) - Z1).abs().amax(dim=1) / scale).max().item()
    assert e3 < 1e-4 and et < 2e-2, (e3, et)
    h.close()


def test_adjoint_directional_derivative_on_128x128_with_viscosity():
    """The viscosity gradient in bench's adjoint configuration (TH P3/P2 on
    128^2 with nu_e = exp(N(0, 1/4))): grad . delta equals the central
    difference of the library's own forward solves in a random direction
    (eps = 1e-5, solves to 1e-10; agreement 1e-5)."""
    w = W.workload("th_p3_128x128_nu")
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT, schedule=w.schedule,
                       host_only=1)
    nc = probe.n_cells()
    i0 = probe.info()
    probe.close()
    nu = W.cell_viscosity(nc, w.seed)
    r = np.random.default_rng(6)
    f = torch.tensor(W.nodal_forcing(i0["n_vel_nodes"], 2, w.seed).reshape(-1), device="cuda")
    gu = torch.tensor(r.standard_normal((2, i0["n_vel_nodes"])), device="cuda")
    gp = torch.tensor(r.standard_normal(i0["n_pres_nodes"]), device="cuda")

    def forward(nu_):
        hh = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, nu_cell=nu_, hierarchy=P.HIER_EXPLICIT,
                        schedule=w.schedule, precision=P.MIXED)
        u, p, _, rel = hh.solve(f, tol=1e-10)
        assert rel <= 1e-10
        return hh, u, p

    h, u, p = forward(nu)
    lam_u, _, _, _, arel = h.adjoint(gu, gp, tol=1e-10)
    assert arel <= 1e-10
    g = h.grad_viscosity(u, lam_u).cpu().numpy()
    h.close()
    dn = r.standard_normal(nc) * nu
    eps = 1e-5
    L = []
    for sgn in (1, -1):
        hh, uu, pp = forward(nu + sgn * eps * dn)
        L.append(float((gu.reshape(-1) * uu).sum() + (gp * pp).sum()))
        hh.close()
    fd = (L[0] - L[1]) / (2 * eps)
    an = float(g @ dn)
    assert abs(fd - an) <= 1e-5 * max(abs(an), 1.0), (fd, an)


def test_bench_relaxation_iterations_stay_flat_under_refinement():
    """The bench's relaxation (Chebyshev of degree 2 on [0.5, 2.0] lambda_max
    from 8 Arnoldi steps, pre and post): FGMRES-phMG on TH P4/P3 needs about
    as many iterations on 128^2 as on 64^2 (measured 9 and 11; 12 on 256^2),
    where the degree-1 default needs 20 and 30 (81 on 256^2)."""
    from bench import RELAX
    v, c = W.unit_square_mesh(8)
    its = []
    for nref in (3, 4):
        h = P.StokesMG(v, c, nref, P.TH, 4, hierarchy=P.HIER_EXPLICIT, schedule=[4, 2], precision=P.MIXED,
                       **RELAX["v22"])
        nV = h.info()["n_vel_nodes"]
        f = torch.tensor(W.nodal_forcing(nV, 2, 0).reshape(-1), device="cuda")
        _, _, it, rel = h.solve(f, tol=1e-8)
        assert rel <= 1e-8
        its.append(it)
        h.close()
    assert its[0] <= 11 and its[1] <= its[0] + 3, its


def test_batched_forward_and_adjoint_on_128x128_as_bench_runs_them():
    """The bench's 32-forcing batch on TH P3/P2 128^2 with nu_e = exp(N(0, 1/4))
    (stokes_solve_batched, stokes_adjoint_solve_batched and
    stokes_grad_viscosity_batched, 3xTF32 batched V-cycle, tolerance 1e-8):
    sampled columns have a true relative residual <= 2e-8 under the oracle's
    independently assembled operator and load (the library stops at 1e-8 on
    its own operator), every column converged, and the batched viscosity
    gradient equals the sum of the columns' single gradients (1e-12)."""
    w = W.workload("th_p3_128x128_nu")
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT, schedule=w.schedule,
                       host_only=1)
    nc = probe.n_cells()
    cent = probe.cell_centroids()
    probe.close()
    nu_l = W.cell_viscosity(nc, w.seed)
    meshes, _ = geometry.hierarchy(w.verts, w.cells, w.n_refine, False)
    vf, cf = meshes[0]
    pc = permutation(keys(cent, np.zeros(nc)), keys(vf[cf].mean(axis=1), np.zeros(len(cf))))
    nu_o = nu_l[pc]                                   # oracle cell i is library cell pc[i]
    D = stokes.discretize(vf, cf, stokes.TH, w.k, nu_cells=nu_o)
    h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, nu_cell=nu_l, hierarchy=P.HIER_EXPLICIT,
                   schedule=w.schedule, precision=P.MIXED)
    pv, pq = full_field_perms(h, D)
    nV, d, nb = D.V.n, D.d, 32
    F_l = np.stack([W.nodal_forcing(nV, d, w.seed + 100 + q) for q in range(nb)])     # library node order
    U, Pp, its, rel = h.solve_batched(torch.tensor(F_l.reshape(nb, -1), device="cuda"), tol=1e-8)
    assert np.all(rel <= 1e-8), rel
    for q in (0, 13, 31):
        f_o = F_l[q][:, pv]                          # the same forcing in the oracle's node order
        b, _ = stokes.load_vector(D, f_o)
        u_o = U[q].cpu().numpy().reshape(d, -1)[:, pv].reshape(-1)
        x = np.concatenate([u_o, Pp[q].cpu().numpy()[pq]])[D.free]
        res = np.linalg.norm(b - D.K @ x) / np.linalg.norm(b)
        assert res <= 2e-8, (q, res)
    ut = torch.tensor(np.random.default_rng(w.seed + 9).uniform(-1.0, 1.0, (d, nV)).reshape(-1), device="cuda")
    GU = (U - ut).contiguous()
    GP = torch.zeros_like(Pp)
    LU, _, _, _, arel = h.adjoint_batched(GU, GP, tol=1e-8)
    assert np.all(arel <= 1e-8), arel
    g = h.grad_viscosity_batched(U, LU)
    ref = sum(h.grad_viscosity(U[q].contiguous(), LU[q].contiguous()) for q in range(nb))
    assert float((g - ref).abs().max() / ref.abs().max()) < 1e-12
    h.close()
