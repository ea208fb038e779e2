"""Parity at the workloads' full sizes, in the launch configuration that
bench.py times (HIER_EXPLICIT schedule, defaults otherwise).

* TH P4/P3 on the 64x64 square (167,299 free DoFs, the benchmark workload):
  lambda_max of every level from the library's SplitMix64 start vector (FP64
  handle 1e-9; the mixed handle's FP32 operator within 1e-4), one
  V-cycle in FP64 (1e-10) and in mixed precision (2e-4) against the oracle's
  V-cycle with the same lambda_max, FGMRES iteration counts (+-1).
* SV P4/P3disc on the Alfeld-refined Delaunay disk and TH P3/P2 on the 16^3
  Kuhn cube: the library's solution, mapped to the oracle's DoFs, has a true
  relative residual <= 2e-8 under the oracle's independently assembled
  operator and load (the solver stops at 1e-8 on its own operator; the two
  operators differ by rounding), and sampled patch inverses match
  numpy.linalg.inv of the oracle's blocks.
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


def test_benchmark_workload_th_p4_64x64():
    w = W.workload("th_p4_64x64")
    ora = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule, lmax=[1.0] * 16)
    h64 = _lib(w, P.FP64)
    hmx = _lib(w, P.MIXED)
    perms = [level_perm(h64, li, L.disc) for li, L in enumerate(ora.levels)]
    lm = h64.info()["lmax"]
    # mixed mode applies M^{-1} K in FP32 inside the FP64-orthogonalised Arnoldi
    for a, b in zip(hmx.info()["lmax"][:len(lm) - 1], lm[:len(lm) - 1]):
        assert abs(a - b) <= 1e-4 * b, (a, b)
    for li, L in enumerate(ora.levels[:-1]):
        v0 = rng.uniform_pm1(0, li, perms[li])
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, mg.Options().eig_steps)
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
