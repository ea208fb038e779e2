"""The batched forward and adjoint solves (stokes_solve_batched,
stokes_adjoint_solve_batched, stokes_grad_viscosity_batched and the batched
torch.autograd wrapper) against the FP64 oracle (oracle/adjoint.py).

Every case has a seeded per-cell viscosity nu_e = exp(N(0, 1/4)) on the
finest mesh and nrhs load cases, each with its own nodal forcing, Dirichlet
data and loss gradient (gu_q, gp_q); the loss of the batch is the sum of the
columns' losses L_q = gu_q . u_q + gp_q . p_q, so dL/dnu is the sum of the
columns' viscosity gradients.

Tolerances: the batched FGMRES stops every column at 1e-12 relative
residual on the library's FP64 operator (the preconditioner is the 3xTF32
batched V-cycle; it changes the iterates, not the solution reached), and the
oracle solves directly, so the columns agree with the oracle as the single
FP64 solves do (1e-9 velocity, 1e-8 pressure and adjoint state, 1e-7 for the
bilinear gradients).  A batch of one reproduces stokes_grad_viscosity bit
for bit (the same per-cell arithmetic); wider batches sum the columns inside
each cell's warp, so they agree with the sum of single-column gradients to
rounding (1e-12).
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, geometry, stokes
from tests.dofmap import full_field_perms, keys, permutation

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")
from paper_2407_07253_gb300 import autograd as PA  # noqa: E402

pytestmark = pytest.mark.gpu

# name: (mesh, n_refine, family, k, schedule, barycentric)
CASES = {
    "th_p3_8x8": (W.unit_square_mesh(2), 2, stokes.TH, 3, [3, 2], False),
    "sv_p3_alfeld": (W.unit_square_mesh(2), 2, stokes.SV, 3, [3, 2], True),
    "th3d_p3": (W.kuhn_cube_mesh(2), 1, stokes.TH, 3, [3, 2], False),
}
TOL = 1e-12
NRHS = 3
_cache = {}


def _setup(name):
    if name in _cache:
        return _cache[name]
    (v, c), nref, fam, k, sched, bary = CASES[name]
    meshes, _ = geometry.hierarchy(v, c, nref, bary)
    vf, cf = meshes[0]
    rng = np.random.default_rng(12)
    nu_o = np.exp(0.5 * rng.standard_normal(len(cf)))
    probe = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, host_only=1)
    cent = probe.cell_centroids()
    probe.close()
    pc = permutation(keys(cent, np.zeros(len(cent))), keys(vf[cf].mean(axis=1), np.zeros(len(cf))))
    nu_l = np.empty_like(nu_o)
    nu_l[pc] = nu_o
    kw = dict(barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, precision=P.MIXED)
    h = P.StokesMG(v, c, nref, fam, k, nu_cell=nu_l, **kw)
    D = stokes.discretize(vf, cf, fam, k, nu_cells=nu_o)
    pv, pq = full_field_perms(h, D)
    d, nV, nQ = D.d, D.V.n, D.Q.n
    F_o = rng.uniform(-1, 1, (NRHS, d, nV))
    G_o = rng.uniform(-1, 1, (NRHS, d, nV))
    GU_o = rng.standard_normal((NRHS, d, nV))
    GP_o = rng.standard_normal((NRHS, nQ))
    _cache[name] = dict(h=h, D=D, pv=pv, pq=pq, pc=pc, nu_o=nu_o, nu_l=nu_l, F_o=F_o, G_o=G_o, GU_o=GU_o, GP_o=GP_o,
                        mesh=(v, c, nref, fam, k), kw=kw)
    return _cache[name]


def _to_lib_v(X_o, pv):
    """[nrhs, d, nV] oracle node order -> device [nrhs, d * nV] library order."""
    X = np.empty_like(X_o)
    X[..., pv] = X_o
    return torch.tensor(X.reshape(X_o.shape[0], -1), device="cuda")


def _to_lib_q(X_o, pq):
    X = np.empty_like(X_o)
    X[..., pq] = X_o
    return torch.tensor(X, device="cuda")


def _from_lib_v(X, pv, d):
    return X.cpu().numpy().reshape(X.shape[0], d, -1)[..., pv]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _run(S, mode=P.BATCH_3XTF32):
    h, D = S["h"], S["D"]
    d = D.d
    U, Pp, _, rel = h.solve_batched(_to_lib_v(S["F_o"], S["pv"]), _to_lib_v(S["G_o"], S["pv"]), mode=mode, tol=TOL)
    assert np.all(rel <= TOL), rel
    LU, LP, GF, _, arel = h.adjoint_batched(_to_lib_v(S["GU_o"], S["pv"]), _to_lib_q(S["GP_o"], S["pq"]), mode=mode,
                                            tol=TOL)
    assert np.all(arel <= TOL), arel
    GN = h.grad_viscosity_batched(U, LU)
    return U, Pp, LU, LP, GF, GN


@pytest.mark.parametrize("name", list(CASES))
def test_batched_forward_adjoint_and_gradients_match_oracle(name):
    S = _setup(name)
    D = S["D"]
    d, nV = D.d, D.V.n
    U, Pp, LU, _, GF, GN = _run(S)
    Uo = _from_lib_v(U, S["pv"], d)
    Po = Pp.cpu().numpy()[:, S["pq"]]
    LUo = _from_lib_v(LU, S["pv"], d)
    GFo = _from_lib_v(GF, S["pv"], d)
    gnu_sum = np.zeros(len(S["nu_o"]))
    for q in range(NRHS):
        x = adjoint.forward(D, S["F_o"][q], S["G_o"][q])
        lam, gf, gnu = adjoint.gradients(D, x, S["GU_o"][q], S["GP_o"][q])
        gnu_sum += gnu
        assert _rel(Uo[q], x[:d * nV].reshape(d, nV)) < 1e-9, q
        assert _rel(Po[q], x[d * nV:]) < 1e-8, q
        assert _rel(LUo[q], lam[:d * nV].reshape(d, nV)) < 1e-8, q
        assert np.all(LUo[q][D.dirichlet[:d * nV].reshape(d, nV)] == 0.0)
        assert _rel(GFo[q], gf) < 1e-7, q
    assert _rel(GN.cpu().numpy()[S["pc"]], gnu_sum) < 1e-7


def test_batched_viscosity_gradient_is_the_sum_of_single_columns():
    S = _setup("th_p3_8x8")
    h = S["h"]
    U, _, LU, _, _, GN = _run(S)
    singles = [h.grad_viscosity(U[q], LU[q]) for q in range(NRHS)]
    assert torch.equal(h.grad_viscosity_batched(U[:1], LU[:1]), singles[0])
    ref = sum(singles)
    assert float((GN - ref).abs().max() / ref.abs().max()) < 1e-12


def test_batched_tf32_preconditioner_reaches_the_same_solution():
    """TF32 products in the V-cycle change the iteration count, not the
    solution the FP64 Krylov iteration converges to."""
    S = _setup("sv_p3_alfeld")
    D = S["D"]
    d, nV = D.d, D.V.n
    U, Pp, _, _, _, _ = _run(S, P.BATCH_TF32)
    Uo = _from_lib_v(U, S["pv"], d)
    for q in range(NRHS):
        x = adjoint.forward(D, S["F_o"][q], S["G_o"][q])
        assert _rel(Uo[q], x[:d * nV].reshape(d, nV)) < 1e-9, q


def test_batched_autograd_matches_direct_calls_and_finite_differences():
    S = _setup("th_p3_8x8")
    v, c, nref, fam, k = S["mesh"]
    kw = dict(S["kw"])
    D = S["D"]
    d = D.d
    F = _to_lib_v(S["F_o"], S["pv"]).view(NRHS, d, -1).clone().requires_grad_(True)
    nu = torch.tensor(S["nu_l"], dtype=torch.float64, requires_grad=True)
    GU = _to_lib_v(S["GU_o"], S["pv"]).view(NRHS, d, -1)
    GP = _to_lib_q(S["GP_o"], S["pq"])
    U, Pp = PA.solve_batched(v, c, nref, fam, k, F, nu, tol=TOL, **kw)
    L = (GU * U).sum() + (GP * Pp).sum()
    L.backward()
    h = P.StokesMG(v, c, nref, fam, k, nu_cell=S["nu_l"], **kw)
    U2, P2, _, _ = h.solve_batched(F.detach().reshape(NRHS, -1), tol=TOL)
    LU, _, GF2, _, _ = h.adjoint_batched(GU.reshape(NRHS, -1), GP, tol=TOL)
    gnu2 = h.grad_viscosity_batched(U2, LU)
    assert torch.equal(U.detach().reshape(NRHS, -1), U2) and torch.equal(Pp.detach(), P2)
    assert torch.equal(F.grad.reshape(NRHS, -1), GF2)
    assert torch.equal(nu.grad.to(gnu2.device), gnu2)
    h.close()
    rng = np.random.default_rng(4)
    dn = torch.tensor(rng.standard_normal(len(S["nu_l"])) * S["nu_l"], dtype=torch.float64)
    eps = 1e-5

    def Lof(nu_):
        with torch.no_grad():
            uu, pp = PA.solve_batched(v, c, nref, fam, k, F.detach(), nu_, tol=TOL, **kw)
            return float((GU * uu).sum() + (GP * pp).sum())
    fd = (Lof(nu.detach() + eps * dn) - Lof(nu.detach() - eps * dn)) / (2 * eps)
    an = float((nu.grad * dn).sum())
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)


def test_batched_solve_arguments_are_checked():
    S = _setup("th_p3_8x8")
    h, D = S["h"], S["D"]
    nv = D.d * D.V.n
    F = torch.zeros(2, nv, dtype=torch.float64, device="cuda")
    for kw in (dict(tol=-1.0), dict(nu=0.0), dict(mode=5)):
        with pytest.raises(P.StokesError) as e:
            h.solve_batched(F, **kw)
        assert e.value.code == -1
    with pytest.raises(P.StokesError) as e:
        h.solve_batched(torch.zeros(P.BATCH_MAX + 1, nv, dtype=torch.float64, device="cuda"))
    assert e.value.code == -1
    v, c, nref, fam, k = S["mesh"]
    h64 = P.StokesMG(v, c, nref, fam, k, hierarchy=P.HIER_EXPLICIT, schedule=[3, 2], precision=P.FP64)
    with pytest.raises(P.StokesError) as e:
        h64.solve_batched(F)
    assert e.value.code == -1
    h64.close()
    # zero forcings and zero Dirichlet data: zero solutions in no iterations
    U, Pp, its, _ = h.solve_batched(F, tol=TOL)
    assert its == 0 and not U.any() and not Pp.any()
