"""Pins of the oracle's discrete adjoint (oracle/adjoint.py).

The gradients are checked against what fixes them independently of the
adjoint formulas:
  * central finite differences of the forward map (bordered direct solves)
    in single cell viscosities, a random viscosity direction and a random
    forcing direction (eps = 1e-6; the maps are smooth, so the error is
    O(eps^2) plus solver rounding);
  * the forcing map is linear: its derivative times a direction equals the
    forward response to that direction exactly (up to rounding);
  * K is symmetric, which the adjoint relies on (K^T lambda = K lambda);
  * the adjoint right-hand side is orthogonal to the pressure constants
    (the null space of K), so the singular system is consistent.
A dropped lifting term, a wrong sign, a transposed element matrix or a
missing mean projection each fails one of these: the cases carry Dirichlet
data, per-cell viscosities and a loss on the pressure.
"""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint, geometry, stokes


def _problem(fam, k, n, d, seed):
    if d == 2:
        v, c = W.unit_square_mesh(n)
    else:
        v, c = W.kuhn_cube_mesh(n)
    if fam == stokes.SV:
        v, c, _ = geometry.refine_alfeld(v, c)
    rng = np.random.default_rng(seed)
    nu = np.exp(0.5 * rng.standard_normal(len(c)))
    return v, c, nu, rng


def _loss_parts(disc, rng):
    d, nV, nQ = disc.d, disc.V.n, disc.Q.n
    gu = rng.standard_normal((d, nV))
    gp = rng.standard_normal(nQ)
    f = rng.uniform(-1, 1, (d, nV))
    g = rng.uniform(-1, 1, (d, nV))          # only boundary values are used
    return gu, gp, f, g


def _loss(disc, x_full, gu, gp):
    d, nV = disc.d, disc.V.n
    return float(gu.reshape(-1) @ x_full[:d * nV] + gp @ x_full[d * nV:])


CASES = [(stokes.TH, 2, 2, 2, 0), (stokes.TH, 3, 2, 2, 1), (stokes.SV, 2, 2, 2, 2), (stokes.TH, 2, 2, 3, 3)]


@pytest.mark.parametrize("fam,k,n,d,seed", CASES)
def test_viscosity_gradient_matches_central_differences(fam, k, n, d, seed):
    v, c, nu, rng = _problem(fam, k, n, d, seed)
    D = stokes.discretize(v, c, fam, k, nu_cells=nu)
    gu, gp, f, g = _loss_parts(D, rng)
    x = adjoint.forward(D, f, g)
    _, _, gnu = adjoint.gradients(D, x, gu, gp)
    eps = 1e-6

    def L(nu_):
        Dp = stokes.discretize(v, c, fam, k, nu_cells=nu_)
        return _loss(Dp, adjoint.forward(Dp, f, g), gu, gp)

    cells = rng.choice(len(c), size=3, replace=False)
    for e in cells:
        dn = np.zeros(len(c)); dn[e] = eps * nu[e]
        fd = (L(nu + dn) - L(nu - dn)) / (2 * eps * nu[e])
        assert abs(fd - gnu[e]) <= 1e-6 * max(1.0, np.abs(gnu).max()), (e, fd, gnu[e])
    direction = rng.standard_normal(len(c)) * nu
    fd = (L(nu + eps * direction) - L(nu - eps * direction)) / (2 * eps)
    assert abs(fd - gnu @ direction) <= 1e-6 * np.abs(gnu).sum() * np.abs(direction).max()


@pytest.mark.parametrize("fam,k,n,d,seed", CASES)
def test_forcing_gradient_is_exact_linear_response(fam, k, n, d, seed):
    v, c, nu, rng = _problem(fam, k, n, d, seed)
    D = stokes.discretize(v, c, fam, k, nu_cells=nu)
    gu, gp, f, g = _loss_parts(D, rng)
    x = adjoint.forward(D, f, g)
    _, gf, _ = adjoint.gradients(D, x, gu, gp)
    df = rng.standard_normal(f.shape)
    # the response of the loss to df alone (g = 0): the map f -> x is linear
    dx = adjoint.forward(D, df, None)
    assert np.isclose(_loss(D, dx, gu, gp), float((gf * df).sum()), rtol=1e-9, atol=1e-12)
    # central differences agree too (the loss is affine in f)
    eps = 1e-3
    fd = (_loss(D, adjoint.forward(D, f + eps * df, g), gu, gp)
          - _loss(D, adjoint.forward(D, f - eps * df, g), gu, gp)) / (2 * eps)
    assert np.isclose(fd, float((gf * df).sum()), rtol=1e-8, atol=1e-12)


def test_operator_symmetric_and_adjoint_rhs_consistent():
    v, c, nu, rng = _problem(stokes.TH, 3, 2, 2, 5)
    D = stokes.discretize(v, c, stokes.TH, 3, nu_cells=nu)
    assert abs(D.K - D.K.T).max() < 1e-13
    gu, gp, _, _ = _loss_parts(D, rng)
    r = adjoint.adjoint_rhs(D, gu, gp)
    pm = D.pressure_mask_free()
    assert abs(r[pm].sum()) < 1e-12 * np.abs(gp).sum()
    lam = adjoint.adjoint(D, gu, gp)
    # K lambda = r on the free DoFs, and lambda vanishes on the Dirichlet DoFs
    assert np.abs(D.K @ lam[D.free] - r).max() < 1e-9 * np.abs(r).max()
    assert np.all(lam[D.dirichlet] == 0.0)


def test_unit_viscosity_gradient_is_minus_the_energy_pairing():
    """Closed form: with nu = 1 and lambda = u (both zero on the boundary),
    the element pairings -lambda_e^T A_e u_e sum to -u^T A u, because the
    cells' matrices assemble to the vector Laplacian A."""
    v, c = W.unit_square_mesh(2)
    D = stokes.discretize(v, c, stokes.TH, 2)
    rng = np.random.default_rng(9)
    x = np.zeros(D.n_full)
    x[:2 * D.V.n] = rng.standard_normal(2 * D.V.n)
    lam = x.copy()
    lam[D.dirichlet] = 0.0
    x[D.dirichlet] = 0.0
    g = adjoint.grad_viscosity(D, x, lam)
    A = D.Kfull[:2 * D.V.n, :2 * D.V.n]
    u = x[:2 * D.V.n]
    assert np.isclose(g.sum(), -(u @ (A @ u)), rtol=1e-12)
