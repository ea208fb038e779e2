"""The batched V-cycle (stokes_mg_vcycle_batched) against the FP64 oracle.

The batch runs the same cycle as the single-vector mixed-precision V-cycle
(Eq. 3.2 / 3.1 with Chebyshev-accelerated ASM relaxation, Sec. 3.3), with the
right-hand sides interleaved DoF-major, SpMM for the SpMVs and transfers and
the patch apply W_i K_i^{-1} R_i as a tensor-core GEMM per patch.

Tolerances:
  * 3xTF32 splits every FP32 operand into a TF32 head and tail and keeps the
    three cross products (on tcgen05 for patches of 65 to 768 DoFs, on the
    warp-level MMA otherwise), which is FP32 accuracy up to the dropped lo*lo
    term (2^-22 relative), so the batch agrees with the oracle to the same
    2e-4 as the single-vector mixed V-cycle (FP32 accumulation over a
    V-cycle), and with that V-cycle itself to 1e-4;
  * TF32 rounds the inverses and residuals to 10 mantissa bits (2^-11
    relative per product), so one V-cycle lands within 2e-2 of the oracle.
Each column of a batch is computed with the same arithmetic in the same
order whatever the width, so the first columns of a wide batch equal a
narrow batch bit for bit, and repeated runs are bitwise equal.
"""
import numpy as np
import pytest

from tests.test_gpu_parity import CASES, from_lib, pair, relerr, to_lib

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

NAMES = ["th_p2_8x8", "th_p4_8x8", "th_p4_gradual", "sv_p3_alfeld", "th3d_p3"]
assert all(n in CASES for n in NAMES)


def _batch(ora, perm, nrhs, seed):
    n = ora.levels[0].disc.n_free
    R_o = np.random.default_rng(seed).standard_normal((nrhs, n))
    R = torch.stack([to_lib(R_o[q], perm) for q in range(nrhs)])
    return R_o, R


@pytest.mark.parametrize("name", NAMES)
def test_batched_3xtf32_matches_oracle_and_single_vcycle(name):
    h, ora, perms = pair(name, P.MIXED)
    R_o, R = _batch(ora, perms[0], 5, 3)
    Z = h.vcycle_batched(R, P.BATCH_3XTF32)
    Z1 = h.vcycle(R)
    for q in range(R.shape[0]):
        z = from_lib(Z[q], perms[0])
        assert relerr(z, ora.vcycle(R_o[q])) < 2e-4, q
        assert relerr(z, from_lib(Z1[q], perms[0])) < 1e-4, q


@pytest.mark.parametrize("name", NAMES)
def test_batched_tf32_matches_oracle(name):
    h, ora, perms = pair(name, P.MIXED)
    R_o, R = _batch(ora, perms[0], 3, 4)
    Z = h.vcycle_batched(R, P.BATCH_TF32)
    for q in range(R.shape[0]):
        assert relerr(from_lib(Z[q], perms[0]), ora.vcycle(R_o[q])) < 2e-2, q


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_columns_independent_of_width_and_deterministic(mode):
    h, ora, perms = pair("th_p4_8x8", P.MIXED)
    _, R = _batch(ora, perms[0], P.BATCH_MAX, 9)
    Zw = h.vcycle_batched(R, mode)                   # width 64
    assert torch.equal(Zw, h.vcycle_batched(R, mode))
    for nrhs in (1, 8, 13, 32):                      # widths 8, 8, 16, 32
        Zn = h.vcycle_batched(R[:nrhs], mode)
        assert torch.equal(Zn, Zw[:nrhs]), nrhs


def test_batched_graph_and_eager_paths_agree():
    h, ora, perms = pair("th_p4_gradual", P.MIXED)
    he, _, _ = pair("th_p4_gradual", P.MIXED, use_graph=0)
    _, R = _batch(ora, perms[0], 20, 6)
    for mode in (P.BATCH_TF32, P.BATCH_3XTF32):
        assert torch.equal(h.vcycle_batched(R, mode), he.vcycle_batched(R, mode))


def test_batched_bad_arguments():
    h, ora, perms = pair("th_p2_8x8", P.MIXED)
    n = ora.levels[0].disc.n_free
    R = torch.zeros(P.BATCH_MAX + 1, n, dtype=torch.float64, device="cuda")
    with pytest.raises(P.StokesError) as e:
        h.vcycle_batched(R)
    assert e.value.code == -1
    with pytest.raises(P.StokesError) as e:
        h.vcycle_batched(R[:2], mode=7)
    assert e.value.code == -1
    h64, _, _ = pair("th_p2_8x8", P.FP64)
    with pytest.raises(P.StokesError) as e:
        h64.vcycle_batched(R[:2])
    assert e.value.code == -1


def _consistent_rhs(ora, nrhs, seed):
    """Random free-DoF right-hand sides with mean-free pressure parts (the
    consistency condition of the singular all-Dirichlet system, Sec. 2)."""
    D = ora.levels[0].disc
    B = np.random.default_rng(seed).standard_normal((nrhs, D.n_free))
    pm = D.pressure_mask_free()
    B[:, pm] -= B[:, pm].mean(axis=1, keepdims=True)
    return B


@pytest.mark.parametrize("name", ["th_p4_8x8", "sv_p3_alfeld", "th3d_p3"])
def test_batched_fgmres_matches_single_solves(name):
    """stokes_fgmres_batched with the 3xTF32 preconditioner: every column's
    true residual under the oracle's operator is <= 2e-10 (the solve stops at
    1e-10 on the library's operator), and the batch needs the single-RHS
    mixed solver's iteration count within one (the preconditioners agree to
    ~1e-5); repeated runs are bitwise equal."""
    h, ora, perms = pair(name, P.MIXED)
    D = ora.levels[0].disc
    B_o = _consistent_rhs(ora, 5, 8)
    B = torch.stack([to_lib(B_o[q], perms[0]) for q in range(5)])
    X, its, rel = h.fgmres_batched(B, P.BATCH_3XTF32, tol=1e-10)
    assert np.all(rel <= 1e-10), rel
    X2, _, _ = h.fgmres_batched(B, P.BATCH_3XTF32, tol=1e-10)
    assert torch.equal(X, X2)
    its_single = []
    for q in range(5):
        x_o = from_lib(X[q], perms[0])
        res = np.linalg.norm(B_o[q] - D.K @ x_o) / np.linalg.norm(B_o[q])
        assert res <= 2e-10, (q, res)
        its_single.append(h.fgmres(B[q].clone(), tol=1e-10)[1])
    assert abs(its - max(its_single)) <= 1, (its, its_single)


def test_batched_fgmres_tf32_and_widths():
    """TF32 preconditioning still reaches the tolerance (a preconditioner
    need not be accurate; FP64 Krylov arithmetic sets the accuracy), at
    widths 8 and 64."""
    h, ora, perms = pair("th_p4_gradual", P.MIXED)
    D = ora.levels[0].disc
    for nrhs in (3, 64):
        B_o = _consistent_rhs(ora, nrhs, 9)
        B = torch.tensor(np.stack([np.asarray(to_lib(B_o[q], perms[0]).cpu()) for q in range(nrhs)]), device="cuda")
        X, its, rel = h.fgmres_batched(B, P.BATCH_TF32, tol=1e-9)
        assert np.all(rel <= 1e-9), rel
        for q in (0, nrhs - 1):
            x_o = from_lib(X[q], perms[0])
            res = np.linalg.norm(B_o[q] - D.K @ x_o) / np.linalg.norm(B_o[q])
            assert res <= 2e-9, (nrhs, q, res)


@pytest.mark.parametrize("name", ["sv_p3_alfeld", "th3d_p3", "sv_p4_disk"])
def test_batched_plan_buckets_cover_every_patch_once(name):
    """The autotuned plan of every relaxed level: its launches cover the
    level's patches once, in size order, each launch of one kind (tensor
    cores exactly for the patches of more than 64 DoFs; in 3xTF32 up to 768,
    the largest whose split operands leave two pipeline stages)."""
    h, ora, perms = pair(name, P.MIXED)
    _, R = _batch(ora, perms[0], 8, 2)
    for mode in (P.BATCH_TF32, P.BATCH_3XTF32):
        h.vcycle_batched(R, mode)
        for li in range(h.info()["n_levels"] - 1):
            off, _ = h.patches(li)
            sizes = np.sort(np.diff(off))
            parts, single = h.batch_plan(li, mode)
            assert sum(pt["count"] for pt in parts) == len(sizes) and single > 0
            i = 0
            for pt in parts:
                seg = sizes[i:i + pt["count"]]
                assert seg[0] == pt["lo"] and seg[-1] == pt["hi"], (li, pt)
                tc = pt["lo"] > 64 and (mode == P.BATCH_TF32 or pt["hi"] <= 768)
                assert pt["kind"] == (2 if tc else 1) and (tc or pt["hi"] <= 64 or pt["lo"] > 768), (li, pt)
                assert pt["us"] > 0
                i += pt["count"]


@pytest.mark.parametrize("name", ["sv_p4_disk", "th3d_p3"])
def test_batched_tuned_plan_gives_the_untuned_result(name):
    """A patch's arithmetic depends only on its kind, so the tuned buckets and
    launch shapes give the result of one launch per kind bit for bit."""
    h, ora, perms = pair(name, P.MIXED)
    hu, _, _ = pair(name, P.MIXED, batch_tune=0)
    _, R = _batch(ora, perms[0], 16, 7)
    for mode in (P.BATCH_TF32, P.BATCH_3XTF32):
        assert torch.equal(h.vcycle_batched(R, mode), hu.vcycle_batched(R, mode))
        parts, single = hu.batch_plan(0, mode)
        assert single == 0.0 and len(parts) <= 2


def test_bounded_mbarrier_wait_gives_up_and_returns():
    """The tensor-core kernel's mbarrier waits are bounded: a wait on a barrier
    that nothing arrives on runs out after the given number of polls, sets
    its status and the kernel returns, leaving the context usable."""
    assert P._binding.selftest_bounded_wait(1000) == 2
    assert P._binding.selftest_bounded_wait(100000) == 2
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum()) == 8.0
