"""Pins of the oracle's building blocks against closed forms and textbook
facts (no GPU).  Each test names the property it checks and where it comes
from."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import geometry, lagrange, rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_sequence():
    """SplitMix64 from state 0 reproduces the published output sequence."""
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.startswith("0x")]
    got = [int(v) for v in rng.splitmix64(0, 0, np.arange(3))]
    assert got == want
    u = rng.uniform_pm1(5, 3, np.arange(100000))
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("deg", [0, 2, 5, 8])
def test_quadrature_exact_on_monomials(d, deg):
    """int_ref x^a y^b (z^c) = a! b! c! / (a+b+c+d)!  times d! (weights sum to 1)."""
    lam, w = lagrange.quadrature(d, deg)
    x = lam[:, 1:]
    for a in np.ndindex(*([deg + 1] * d)):
        if sum(a) > deg:
            continue
        exact = math.prod(math.factorial(ai) for ai in a) / math.factorial(sum(a) + d) * math.factorial(d)
        got = np.sum(w * np.prod(x ** np.array(a), axis=1))
        assert abs(got - exact) < 1e-14, (a, got, exact)


@pytest.mark.parametrize("d,k", [(2, 1), (2, 2), (2, 4), (2, 7), (3, 1), (3, 3), (3, 4)])
def test_lagrange_nodal_and_reproduction(d, k):
    """phi_alpha(node_beta) = delta; sum phi = 1; the interpolant of any
    polynomial of degree k reproduces it; gradients match central
    differences of the values."""
    al = np.array(lagrange.multi_indices(k, d), dtype=float)
    assert len(al) == math.comb(k + d, d)
    nodes = al / k
    V = lagrange.basis(k, d, nodes)
    assert np.allclose(V, np.eye(len(al)), atol=1e-13)
    r = np.random.default_rng(1)
    pts = r.dirichlet(np.ones(d + 1), size=50)
    B = lagrange.basis(k, d, pts)
    assert np.allclose(B.sum(1), 1.0, atol=1e-12)
    coef = r.normal(size=len(al))
    expo = al[:, 1:].astype(int)
    poly = lambda x: (coef[None] * np.prod(x[:, None, :] ** expo[None], axis=2)).sum(1)  # noqa: E731
    assert np.allclose(B @ poly(nodes[:, 1:]), poly(pts[:, 1:]), atol=1e-10)
    # gradient in cartesian reference coordinates vs central differences
    D = lagrange.basis_dlam(k, d, pts)
    gref = D[:, :, 1:] - D[:, :, :1]
    h = 1e-6
    for j in range(d):
        e = np.zeros(d + 1); e[j + 1] = h; e[0] = -h
        fd = (lagrange.basis(k, d, pts + e) - lagrange.basis(k, d, pts - e)) / (2 * h)
        assert np.allclose(gref[:, :, j], fd, atol=1e-6 * max(1, k ** 2))


def test_p1_stiffness_is_cotangent_formula():
    """P1 stiffness on a triangle: S_ij = -cot(theta_k)/2 for i != j."""
    from oracle import stokes
    v = np.array([[0.0, 0.0], [2.0, 0.1], [0.3, 1.2]])
    c = np.array([[0, 1, 2]])
    S, M, C, vol = stokes.element_matrices(v, c, 1, 0, 2)
    S = S[0]
    for i, j, k in [(0, 1, 2), (1, 2, 0), (0, 2, 1)]:
        a, b = v[i] - v[k], v[j] - v[k]
        cot = np.dot(a, b) / abs(a[0] * b[1] - a[1] * b[0])
        assert abs(S[i, j] + cot / 2) < 1e-14
    assert np.allclose(S.sum(1), 0, atol=1e-14)
    # P1 mass: |T|/12 (1 + delta_ij)
    assert np.allclose(M[0], vol[0] / 12 * (np.ones((3, 3)) + np.eye(3)), atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_uniform_refinement_nested(d):
    """R_u keeps total volume, multiplies cells by 2^d, and every child lies
    inside its parent (barycentric coordinates of its vertices in [0,1])."""
    v, c = (W.unit_square_mesh(2) if d == 2 else W.kuhn_cube_mesh(1))
    vf, cf, par = geometry.refine_uniform(v, c)
    assert len(cf) == len(c) * 2 ** d
    vol_c = geometry.cell_volumes(v, c)
    vol_f = geometry.cell_volumes(vf, cf)
    assert abs(vol_f.sum() - vol_c.sum()) < 1e-13
    assert np.allclose(np.bincount(par, weights=vol_f), vol_c, atol=1e-14)
    for fc in range(len(cf)):
        lam = lagrange.to_barycentric(v, c[par[fc]], vf[cf[fc]])
        assert lam.min() > -1e-12 and lam.max() < 1 + 1e-12


def test_square_and_kuhn_refinement_reproduce_structured_meshes():
    """Quadrisection of the n x n mesh is the 2n x 2n mesh; Bey's refinement
    of the Kuhn n^3 mesh is the Kuhn (2n)^3 mesh (same cells as vertex sets)."""
    def key(V, C, s):
        return sorted(tuple(sorted(map(tuple, np.round(V[cc] * s).astype(int).tolist()))) for cc in C)
    v, c = W.unit_square_mesh(3)
    vf, cf, _ = geometry.refine_uniform(v, c)
    assert key(vf, cf, 6) == key(*W.unit_square_mesh(6), 6)
    v, c = W.kuhn_cube_mesh(2)
    vf, cf, _ = geometry.refine_uniform(v, c)
    assert key(vf, cf, 4) == key(*W.kuhn_cube_mesh(4), 4)


def test_alfeld_split():
    """R_b: d+1 children per cell sharing the barycenter, same volume."""
    v, c = W.delaunay_disk_mesh(0)
    vf, cf, par = geometry.refine_alfeld(v, c)
    assert len(cf) == 3 * len(c)
    assert np.allclose(np.bincount(par, weights=geometry.cell_volumes(vf, cf)), geometry.cell_volumes(v, c))
    assert len(vf) == len(v) + len(c)


def test_delaunay_disk_workload_size():
    """The seeded disk has ~250 triangles; two R_u steps give ~4k (the
    'about 4k macro-triangles' of the Scott-Vogelius workload)."""
    v, c = W.delaunay_disk_mesh(0)
    assert 200 <= len(c) <= 300
    assert 3200 <= 16 * len(c) <= 4800
    assert geometry.cell_volumes(v, c).min() > 1e-4
