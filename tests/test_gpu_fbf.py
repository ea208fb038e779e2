"""FBF(phMG) (stokes_fbf_setup, Eq. fbf) against the FP64 oracle
(oracle/fbf.py).

Each case is Scott-Vogelius on the Alfeld-refined finest mesh with a
seeded per-cell viscosity.  Checked, with the oracle using the library's
lambda_max values where a single application is compared:
  * lambda_max of every velocity level from the library's SplitMix64 start
    equals the oracle's Arnoldi from the same start (1e-8: the coarse 3D
    velocity level has fewer free nodes than Arnoldi steps, so the last
    columns are near breakdown and carry ~1e-9 of rounding);
  * one scalar velocity V-cycle A~^-1 in FP64 (1e-10) and in mixed precision
    (2e-4, FP32 accumulation over one V-cycle as in the monolithic solver);
  * one FBF application P^-1 r (FP64, 1e-10);
  * the FGMRES-FBF solve: the library's solution equals the oracle's direct
    solution to the solver tolerance, and the iteration count is the
    oracle's FBF-FGMRES count within one.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fbf, geometry, multigrid, rng, stokes
from tests.dofmap import full_field_perms, keys, permutation

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

# name: (mesh, n_refine, k, schedule)
CASES = {
    "sv_p2_4x4": (W.unit_square_mesh(2), 1, 2, [2]),
    "sv_p3_8x8": (W.unit_square_mesh(2), 2, 3, [3, 2]),
    "sv_p4_4x4": (W.unit_square_mesh(2), 1, 4, [4, 2]),
    "sv3d_p3": (W.kuhn_cube_mesh(1), 1, 3, [3, 2]),
}
_cache = {}


def _setup(name, precision=P.FP64):
    key = (name, precision)
    if key in _cache:
        return _cache[key]
    (v, c), nref, k, sched = CASES[name]
    meshes, _ = geometry.hierarchy(v, c, nref, True)
    vf, cf = meshes[0]
    r = np.random.default_rng(5)
    nu_o = np.exp(0.5 * r.standard_normal(len(cf)))
    probe = P.StokesMG(v, c, nref, P.SV, k, fbf=True, hierarchy=P.HIER_EXPLICIT, schedule=sched, host_only=1)
    cent = probe.cell_centroids()
    probe.close()
    pc = permutation(keys(cent, np.zeros(len(cent))), keys(vf[cf].mean(axis=1), np.zeros(len(cf))))
    nu_l = np.empty_like(nu_o)
    nu_l[pc] = nu_o
    ora_lm = fbf.VelocityHierarchy(v, c, nref, sched, barycentric=True, nu_cells=nu_o)
    lm = [L.lmax for L in ora_lm.levels[:-1]]
    h = P.StokesMG(v, c, nref, P.SV, k, fbf=True, nu_cell=nu_l, hierarchy=P.HIER_EXPLICIT, schedule=sched,
                   lmax_override=lm, precision=precision)
    D = stokes.discretize(vf, cf, stokes.SV, k, nu_cells=nu_o)
    # scalar level perms: library free node perm[i] is oracle free node i
    sperm = []
    for li, L in enumerate(ora_lm.levels):
        xyz, comp, _ = h.level_dofs(li)
        ox = L.disc.V.coords[L.disc.free]
        sperm.append(permutation(keys(xyz, comp), keys(ox, np.zeros(len(ox)))))
    pv, pq = full_field_perms(h, D)
    d, nvf = D.d, ora_lm.levels[0].disc.n_free
    # Stokes free order: oracle index i -> library index
    st = np.concatenate([c_ * nvf + sperm[0] for c_ in range(d)] + [d * nvf + pq])
    S = dict(h=h, D=D, vh=ora_lm, sperm=sperm, st=st, pv=pv, pq=pq, nu_o=nu_o, nu_l=nu_l, lm=lm,
             mesh=(v, c, nref, k, sched))
    _cache[key] = S
    return S


def _lib(x_o, perm):
    x = np.empty_like(x_o)
    x[perm] = x_o
    return torch.tensor(x, device="cuda")


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
def test_velocity_lambda_max(name):
    S = _setup(name)
    (v, c), nref, k, sched = CASES[name]
    hd = P.StokesMG(v, c, nref, P.SV, k, fbf=True, nu_cell=S["nu_l"], hierarchy=P.HIER_EXPLICIT, schedule=sched)
    lm = hd.info()["lmax"]
    for li, L in enumerate(S["vh"].levels[:-1]):
        v0 = rng.uniform_pm1(0, li, S["sperm"][li])
        want = multigrid.arnoldi_lmax(L.disc.K, L.asm.apply, v0, multigrid.Options().eig_steps)
        assert abs(lm[li] - want) <= 1e-8 * abs(want), (li, lm[li], want)
    hd.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [P.FP64, P.MIXED])
def test_velocity_vcycle(name, precision):
    S = _setup(name, precision)
    n = S["vh"].levels[0].disc.n_free
    r = np.random.default_rng(1).standard_normal(n)
    z = S["h"].vcycle(_lib(r, S["sperm"][0])).cpu().numpy()[S["sperm"][0]]
    assert _rel(z, S["vh"].vcycle(r)) < (1e-10 if precision == P.FP64 else 2e-4)


@pytest.mark.parametrize("name", list(CASES))
def test_fbf_apply(name):
    S = _setup(name)
    F = fbf.FBF(S["D"], S["vh"], nu_cells=S["nu_o"])
    r = np.random.default_rng(2).standard_normal(S["D"].n_free)
    z = S["h"].fbf_apply(_lib(r, S["st"])).cpu().numpy()[S["st"]]
    assert _rel(z, F.apply(r)) < 1e-10


@pytest.mark.parametrize("name", list(CASES))
def test_fbf_solve(name):
    S = _setup(name)
    D, h = S["D"], S["h"]
    d, nV = D.d, D.V.n
    r = np.random.default_rng(3)
    f_o = r.uniform(-1, 1, (d, nV))
    g_o = r.uniform(-1, 1, (d, nV))

    def lib_v(x):
        y = np.empty_like(x)
        y[:, S["pv"]] = x
        return torch.tensor(y.reshape(-1), device="cuda")
    u, p, its, rel = h.solve(lib_v(f_o), lib_v(g_o), tol=1e-10)
    assert rel <= 1e-10
    b, xD = stokes.load_vector(D, f_o, g_o)
    x = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), xD))
    U = u.cpu().numpy().reshape(d, -1)[:, S["pv"]]
    Pp = p.cpu().numpy()[S["pq"]]
    assert _rel(U, x[:d * nV].reshape(d, nV)) < 1e-7
    assert _rel(Pp, x[d * nV:]) < 1e-6
    F = fbf.FBF(D, S["vh"], nu_cells=S["nu_o"])
    _, its_o, _ = fbf.solve(F, f_o, g_o, tol=1e-10)
    assert abs(its - its_o) <= 1, (its, its_o)


def test_fbf_apply_rejects_a_monolithic_handle():
    v, c = W.unit_square_mesh(2)
    h = P.StokesMG(v, c, 1, P.TH, 2)
    with pytest.raises(P.StokesError) as e:
        h.fbf_apply(torch.zeros(10, dtype=torch.float64, device="cuda"))
    assert e.value.code == -1
    h.close()


@pytest.mark.parametrize("name", ["sv_p3_8x8", "sv3d_p3"])
def test_fbf_mixed_precision(name):
    """Mixed precision (FP32 velocity V-cycles): one application agrees with
    the FP64 oracle to 1e-3 (two V-cycles of ~2e-4 each, composed through B
    and S~^-1), and FGMRES-FBF still reaches the direct solution (5e-7: the
    solver stops on the residual, and the 3D SV system amplifies it by its
    condition number) with the FP64 solver's iteration count within two."""
    S = _setup(name, P.MIXED)
    S64 = _setup(name, P.FP64)
    F = fbf.FBF(S["D"], S["vh"], nu_cells=S["nu_o"])
    r = np.random.default_rng(2).standard_normal(S["D"].n_free)
    z = S["h"].fbf_apply(_lib(r, S["st"])).cpu().numpy()[S["st"]]
    assert _rel(z, F.apply(r)) < 1e-3
    D = S["D"]
    d, nV = D.d, D.V.n
    f_o = np.random.default_rng(3).uniform(-1, 1, (d, nV))

    def lib_v(x):
        y = np.empty_like(x)
        y[:, S["pv"]] = x
        return torch.tensor(y.reshape(-1), device="cuda")
    u, p, its, rel = S["h"].solve(lib_v(f_o), tol=1e-10)
    _, _, its64, _ = S64["h"].solve(lib_v(f_o), tol=1e-10)
    b, xD = stokes.load_vector(D, f_o)
    x = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), xD))
    U = u.cpu().numpy().reshape(d, -1)[:, S["pv"]]
    assert rel <= 1e-10 and _rel(U, x[:d * nV].reshape(d, nV)) < 5e-7
    assert abs(its - its64) <= 2, (its, its64)


def test_fbf_with_hmg_velocity_cycle():
    """FBF(hMG), the paper's other FBF variant: the same entry with the
    hierarchy STOKES_HIER_HMG (no p-coarsening: P_k on every mesh).  One
    application matches the oracle's FBF over the hMG velocity hierarchy, and
    the solve reaches the direct solution."""
    v, c = W.unit_square_mesh(2)
    k, nref = 3, 1
    meshes, _ = geometry.hierarchy(v, c, nref, True)
    D = stokes.discretize(*meshes[0], stokes.SV, k)
    vh = fbf.VelocityHierarchy(v, c, nref, [k], barycentric=True)
    lm = [L.lmax for L in vh.levels[:-1]]
    h = P.StokesMG(v, c, nref, P.SV, k, fbf=True, hierarchy=P.HIER_HMG, lmax_override=lm, precision=P.FP64)
    assert h.info()["n_levels"] == len(vh.levels)
    xyz, comp, _ = h.level_dofs(0)
    ox = vh.levels[0].disc.V.coords[vh.levels[0].disc.free]
    sp0 = permutation(keys(xyz, comp), keys(ox, np.zeros(len(ox))))
    pv, pq = full_field_perms(h, D)
    nvf = vh.levels[0].disc.n_free
    st = np.concatenate([c_ * nvf + sp0 for c_ in range(D.d)] + [D.d * nvf + pq])
    r = np.random.default_rng(4).standard_normal(D.n_free)
    z = h.fbf_apply(_lib(r, st)).cpu().numpy()[st]
    assert _rel(z, fbf.FBF(D, vh).apply(r)) < 1e-10
    f_o = np.random.default_rng(5).uniform(-1, 1, (D.d, D.V.n))
    fl = np.empty_like(f_o)
    fl[:, pv] = f_o
    u, p, its, rel = h.solve(torch.tensor(fl.reshape(-1), device="cuda"), tol=1e-10)
    b, xD = stokes.load_vector(D, f_o)
    x = stokes.zero_mean_pressure(D, stokes.expand(D, stokes.direct_solve(D, b), xD))
    U = u.cpu().numpy().reshape(D.d, -1)[:, pv]
    assert rel <= 1e-10 and _rel(U, x[:D.d * D.V.n].reshape(D.d, D.V.n)) < 1e-7
    h.close()
