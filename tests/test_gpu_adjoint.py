"""The library's discrete adjoint (stokes_adjoint_solve, stokes_grad_viscosity
and the torch.autograd wrapper) against the FP64 oracle (oracle/adjoint.py).

Every case has a seeded per-cell viscosity nu_e = exp(N(0, 1/4)) on the
finest mesh, Dirichlet data on the boundary and a loss with both a velocity
and a pressure part, L = gu . u + gp . p.  The forward solve with variable
viscosity is checked first (setup's nu_cell against the oracle's
discretisation), then the adjoint state, dL/df and dL/dnu.

Tolerances: both sides solve to 1e-12 relative residual (the oracle
directly), so the solutions agree to about kappa(K) * 1e-12; the gradients
are bilinear in (u, lambda), checked to 1e-7 relative to their largest
entry.  The autograd wrapper must reproduce the direct calls exactly, and
its gradient must match a central difference of the library's own forward
solves in a random viscosity direction (eps = 1e-5, agreement 1e-6).
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
    "th_p2_8x8": (W.unit_square_mesh(2), 2, stokes.TH, 2, [2], False),
    "th_p3_8x8": (W.unit_square_mesh(2), 2, stokes.TH, 3, [3, 2], False),
    "sv_p3_alfeld": (W.unit_square_mesh(2), 2, stokes.SV, 3, [3, 2], True),
    "th3d_p3": (W.kuhn_cube_mesh(2), 1, stokes.TH, 3, [3, 2], False),
}
TOL = 1e-12
_cache = {}


def _setup(name):
    if name in _cache:
        return _cache[name]
    (v, c), nref, fam, k, sched, bary = CASES[name]
    meshes, _ = geometry.hierarchy(v, c, nref, bary)
    vf, cf = meshes[0]
    rng = np.random.default_rng(11)
    nu_o = np.exp(0.5 * rng.standard_normal(len(cf)))
    probe = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, host_only=1)
    cent = probe.cell_centroids()
    probe.close()
    # library cell perm[i] is oracle cell i
    pc = permutation(keys(cent, np.zeros(len(cent))), keys(vf[cf].mean(axis=1), np.zeros(len(cf))))
    nu_l = np.empty_like(nu_o)
    nu_l[pc] = nu_o
    h = P.StokesMG(v, c, nref, fam, k, barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, nu_cell=nu_l,
                   precision=P.FP64)
    D = stokes.discretize(vf, cf, fam, k, nu_cells=nu_o)
    pv, pq = full_field_perms(h, D)
    d, nV, nQ = D.d, D.V.n, D.Q.n
    f_o = rng.uniform(-1, 1, (d, nV))
    g_o = rng.uniform(-1, 1, (d, nV))
    gu_o = rng.standard_normal((d, nV))
    gp_o = rng.standard_normal(nQ)
    _cache[name] = dict(h=h, D=D, pv=pv, pq=pq, pc=pc, nu_o=nu_o, nu_l=nu_l, f_o=f_o, g_o=g_o, gu_o=gu_o, gp_o=gp_o,
                        mesh=(v, c, nref, fam, k, sched, bary))
    return _cache[name]


def _to_lib_v(x_o, pv):
    x = np.empty_like(x_o)
    x[:, pv] = x_o
    return torch.tensor(x.reshape(-1), device="cuda")


def _to_lib_q(x_o, pq):
    x = np.empty_like(x_o)
    x[pq] = x_o
    return torch.tensor(x, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _lib_forward_adjoint(S):
    h, D = S["h"], S["D"]
    d = D.d
    u, p, _, rel = h.solve(_to_lib_v(S["f_o"], S["pv"]), _to_lib_v(S["g_o"], S["pv"]), tol=TOL)
    assert rel <= TOL
    lam_u, lam_p, gf, _, arel = h.adjoint(_to_lib_v(S["gu_o"], S["pv"]).view(d, -1), _to_lib_q(S["gp_o"], S["pq"]),
                                          tol=TOL)
    assert arel <= TOL
    gnu = h.grad_viscosity(u, lam_u)
    U = u.cpu().numpy().reshape(d, -1)[:, S["pv"]]
    Pp = p.cpu().numpy()[S["pq"]]
    LU = lam_u.cpu().numpy().reshape(d, -1)[:, S["pv"]]
    GF = gf.cpu().numpy().reshape(d, -1)[:, S["pv"]]
    GN = gnu.cpu().numpy()[S["pc"]]
    return U, Pp, LU, GF, GN


@pytest.mark.parametrize("name", list(CASES))
def test_forward_with_cell_viscosity_matches_oracle(name):
    S = _setup(name)
    D = S["D"]
    U, Pp, _, _, _ = _lib_forward_adjoint(S)
    x = adjoint.forward(D, S["f_o"], S["g_o"])
    d, nV = D.d, D.V.n
    assert _rel(U, x[:d * nV].reshape(d, nV)) < 1e-9
    assert _rel(Pp, x[d * nV:]) < 1e-8


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_state_and_gradients_match_oracle(name):
    S = _setup(name)
    D = S["D"]
    U, Pp, LU, GF, GN = _lib_forward_adjoint(S)
    x = adjoint.forward(D, S["f_o"], S["g_o"])
    lam, gf, gnu = adjoint.gradients(D, x, S["gu_o"], S["gp_o"])
    d, nV = D.d, D.V.n
    assert _rel(LU, lam[:d * nV].reshape(d, nV)) < 1e-8
    assert np.all(LU[D.dirichlet[:d * nV].reshape(d, nV)] == 0.0)
    assert _rel(GF, gf) < 1e-7
    assert _rel(GN, gnu) < 1e-7


def test_autograd_wrapper_matches_direct_calls_and_finite_differences():
    S = _setup("th_p3_8x8")
    v, c, nref, fam, k, sched, bary = S["mesh"]
    D = S["D"]
    d = D.d
    kw = dict(barycentric=bary, hierarchy=P.HIER_EXPLICIT, schedule=sched, precision=P.FP64)
    f = _to_lib_v(S["f_o"], S["pv"]).view(d, -1).clone().requires_grad_(True)
    nu = torch.tensor(S["nu_l"], dtype=torch.float64, requires_grad=True)
    gu = _to_lib_v(S["gu_o"], S["pv"]).view(d, -1)
    gp = _to_lib_q(S["gp_o"], S["pq"])
    u, p = PA.solve(v, c, nref, fam, k, f, nu, tol=TOL, **kw)
    L = (gu * u).sum() + (gp * p).sum()
    L.backward()
    # the same through the direct calls (zero Dirichlet data here)
    h = P.StokesMG(v, c, nref, fam, k, nu_cell=S["nu_l"], **kw)
    u2, p2, _, _ = h.solve(f.detach().reshape(-1), tol=TOL)
    lam_u, _, gf2, _, _ = h.adjoint(gu, gp, tol=TOL)
    gnu2 = h.grad_viscosity(u2, lam_u)
    assert torch.equal(u.detach().reshape(-1), u2) and torch.equal(p.detach(), p2)
    assert torch.equal(f.grad.reshape(-1), gf2.reshape(-1))
    assert torch.equal(nu.grad.to(gnu2.device), gnu2)
    # central difference of the library's own forward solves
    rng = np.random.default_rng(3)
    dn = torch.tensor(rng.standard_normal(len(S["nu_l"])) * S["nu_l"], dtype=torch.float64)
    eps = 1e-5

    def Lof(nu_):
        with torch.no_grad():
            uu, pp = PA.solve(v, c, nref, fam, k, f.detach(), nu_, tol=TOL, **kw)
            return float((gu * uu).sum() + (gp * pp).sum())
    fd = (Lof(nu.detach() + eps * dn) - Lof(nu.detach() - eps * dn)) / (2 * eps)
    an = float((nu.grad * dn).sum())
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1.0), (fd, an)
    h.close()


def test_adjoint_errors_are_reported():
    S = _setup("th_p2_8x8")
    h, D = S["h"], S["D"]
    gu = torch.zeros(D.d, D.V.n, dtype=torch.float64, device="cuda")
    gp = torch.zeros(D.Q.n, dtype=torch.float64, device="cuda")
    for kw in (dict(tol=-1.0), dict(nu=0.0), dict(nu=float("nan"))):
        with pytest.raises(P.StokesError) as e:
            h.adjoint(gu, gp, **kw)
        assert e.value.code == -1
    # a zero loss gradient gives a zero adjoint in no iterations
    lam_u, lam_p, gf, its, _ = h.adjoint(gu, gp, tol=TOL)
    assert its == 0 and not lam_u.any() and not gf.any()
