"""Gradual p-hierarchies at high order (Fig. 7) against the FP64 oracle.

The library builds the hierarchy itself from STOKES_HIER_GRADUAL: k = 6 and 7
go 6/7 -> 4 -> 2, k >= 8 goes k -> 5 -> 2 (the schedule in
tests/golden/pmg_schedule.txt), and Scott-Vogelius levels below the top go
through Taylor-Hood (Sec. 3.2).  The patches are large: up to 561 DoFs at
k = 8 and 758 for SV P6 in 2D, 2,922 for TH P6 and 2,067 for SV P3 in 3D,
which take the saddle inverse's global-memory path.

The patch blocks' condition numbers grow quickly with k on the equispaced
lattice (max over the relaxed levels: 3.0e7 at k = 6, 1.5e8 at k = 7, 8.1e8
at k = 8, against 3.6e6 for the P4 benchmark patches).  The two sides invert
them differently (Schur sweeps here, LAPACK LU in the oracle), so their
inverses agree to about kappa * eps_64, which the V-cycle and lambda_max carry
over.  The FP64 tolerances are therefore max(base, 10 * kappa * eps_64) with
kappa the largest patch condition number of the case (computed from the
oracle's blocks); observed differences are 1e-10 (k = 6), 1.4e-8 (k = 7) and
6e-7 (k = 8), i.e. at most ~3.3 kappa eps_64.

Checks:
  * the level degrees and families equal the schedule;
  * lambda_max of every relaxed level from the library's SplitMix64 start
    equals the oracle's Arnoldi from the same start (base 1e-9);
  * one V-cycle in FP64 (base 1e-10) and mixed precision (2e-4) with the
    same lambda_max;
  * FGMRES to 1e-8: the true residual meets the tolerance and the iteration
    counts agree within one.
"""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg, rng
from tests.dofmap import keys, level_perm, permutation

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

# name: (mesh, n_refine, family, k, expected schedule, barycentric)
CASES = {
    "th_p6_4x4": (W.unit_square_mesh(2), 1, 0, 6, [6, 4, 2], False),
    "th_p7_4x4": (W.unit_square_mesh(2), 1, 0, 7, [7, 4, 2], False),
    "th_p8_4x4": (W.unit_square_mesh(2), 1, 0, 8, [8, 5, 2], False),
    "th_p6_8x8": (W.unit_square_mesh(2), 2, 0, 6, [6, 4, 2], False),
    "sv_p6_alfeld": (W.unit_square_mesh(2), 1, 1, 6, [6, 4, 2], True),
    # 3D (Sec. 4.1.2, Sec. 4.2): Taylor-Hood P6/P5 on the 2^3 Kuhn cube
    # (5,324 free DoFs, patches up to 2,922 DoFs), and monolithic
    # Scott-Vogelius P3/P2disc on its Alfeld split (4,455 free DoFs, patches
    # up to 2,067 DoFs; the coarser levels are Taylor-Hood P2)
    "th3d_p6_2x2x2": (W.kuhn_cube_mesh(2), 0, 0, 6, [6, 4, 2], False),
    "sv3d_p3_alfeld": (W.kuhn_cube_mesh(2), 0, 1, 3, [3, 2], True),
}

_cache = {}


def _pair(name, precision):
    key = (name, precision)
    if key in _cache:
        return _cache[key]
    (v, c), nref, fam, k, sched, bary = CASES[name]
    ora = mg.Hierarchy(v, c, nref, fam, sched, barycentric=bary)
    lm = [L.lmax for L in ora.levels[:-1]]
    h = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_GRADUAL, lmax_override=lm,
                   precision=precision)
    perms = [level_perm(h, li, L.disc) for li, L in enumerate(ora.levels)]
    _cache[key] = (h, ora, perms)
    return _cache[key]


def _kappa_tol(name, base):
    """max(base, 10 kappa eps_64), kappa = largest patch condition number."""
    key = ("kappa", name)
    if key not in _cache:
        _, ora, _ = _pair(name, P.FP64)
        _cache[key] = max(np.linalg.cond(b) for L in ora.levels[:-1] for b in L.asm.blocks)
    return max(base, 10.0 * _cache[key] * np.finfo(np.float64).eps)


def _to_lib(x_o, perm):
    x = np.empty_like(x_o)
    x[perm] = x_o
    return torch.tensor(x, device="cuda")


def _relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("name", list(CASES))
def test_gradual_schedule_levels(name):
    (v, c), nref, fam, k, sched, bary = CASES[name]
    h, ora, _ = _pair(name, P.FP64)
    st = h.info()
    n_p = len(sched) - 1
    assert st["n_levels"] == n_p + nref + 1 + (1 if bary else 0)
    assert list(st["degree"][:n_p + 1]) == sched
    assert all(d == sched[-1] for d in st["degree"][n_p:st["n_levels"]])
    assert st["level_family"][0] == fam
    assert all(f == 0 for f in st["level_family"][1:st["n_levels"]])
    assert list(st["n_free"][:st["n_levels"]]) == [L.disc.n_free for L in ora.levels]


@pytest.mark.parametrize("name", list(CASES))
def test_gradual_lambda_max(name):
    (v, c), nref, fam, k, sched, bary = CASES[name]
    _, ora, perms = _pair(name, P.FP64)
    hd = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_GRADUAL)
    lm = hd.info()["lmax"]
    tol = _kappa_tol(name, 1e-9)
    for li, L in enumerate(ora.levels[:-1]):
        v0 = rng.uniform_pm1(0, li, perms[li])
        want = mg.arnoldi_lmax(L.disc.K, L.asm.apply, v0, mg.Options().eig_steps)
        assert abs(lm[li] - want) <= tol * abs(want), (li, lm[li], want, tol)
    hd.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_gradual_vcycle(name, precision):
    h, ora, perms = _pair(name, precision)
    r = np.random.default_rng(7).standard_normal(ora.levels[0].disc.n_free)
    z = h.vcycle(_to_lib(r, perms[0])).cpu().numpy()[perms[0]]
    err = _relerr(z, ora.vcycle(r))
    tol = _kappa_tol(name, 1e-10) if precision == P.FP64 else 2e-4
    assert err < tol, (err, tol)


@pytest.mark.parametrize("name", list(CASES))
def test_gradual_fgmres(name):
    h, ora, perms = _pair(name, P.FP64)
    D = ora.levels[0].disc
    vx, _, _ = h.nodes()
    pv = permutation(keys(vx, np.zeros(len(vx))), keys(D.V.coords, np.zeros(D.V.n)))
    f_o = W.nodal_forcing(D.V.n, D.d, 0)
    f_l = np.empty_like(f_o)
    f_l[:, pv] = f_o
    _, _, its, rel = h.solve(torch.tensor(f_l.reshape(-1), device="cuda"), tol=1e-8)
    _, its_o, _, _, _ = mg.solve(ora, f_o, None, tol=1e-8)
    assert rel <= 1e-8
    assert abs(its - its_o) <= 1, (its, its_o)
