"""The library's reference tensors (csrc/fem.cpp RefTensors: mass M, stiffness
S[a][b] = int dphi_i/dxi_a dphi_j/dxi_b, coupling Cq[a] = int psi_p dphi_j/dxi_a
and the pressure integrals qint, on the reference simplex of volume 1/d!)
against the oracle's Lagrange basis and quadrature, for TH pairs P_k / P_{k-1}
in 2D up to k = 10 and in 3D up to k = 6.  The device assembly, the load
vector and the zero-mean pressure border all read these tensors; the library
computes them in the Bernstein basis, the oracle by Silvester's product
formula and a conical-product rule.

Tolerance: both sides are float64.  Against a 40-digit evaluation of the
same integrals, the coupling tensor at k = 10 in 2D is off by 1.9e-14
(oracle) and 7.7e-15 (library), relative to its largest entry, so the two
may differ by a few 1e-14; 1e-13 leaves a margin of about three.  (The
earlier monomial construction of the library was off by 3e-5 at k = 10.)"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import lagrange

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("reft") / "reference_tensors_dump")
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-pthread", os.path.join(ROOT, "tests", "reference_tensors_dump.cpp"),
                        os.path.join(ROOT, "paper_2407_07253_gb300", "csrc", "fem.cpp"), "-o", exe],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]

    def run(d, k, points=None):
        if points is not None:
            txt = "\n".join(" ".join(repr(float(x)) for x in p) for p in points) + "\n"
            out = subprocess.run([exe, str(d), str(k), "eval"], input=txt, capture_output=True, text=True,
                                 check=True).stdout.split("\n")
            nb = len(lagrange.multi_indices(k, d))
            av = [tuple(map(int, x.split()))[:d + 1] for x in out[:nb]]
            vals = np.array([[float(y) for y in x.split()] for x in out[nb:] if x])
            return av, vals
        out = subprocess.run([exe, str(d), str(k)], capture_output=True, text=True, check=True).stdout.split("\n")
        nb, nq = map(int, out[0].split())
        av = [tuple(map(int, x.split()))[:d + 1] for x in out[1:1 + nb]]
        aq = [tuple(map(int, x.split()))[:d + 1] for x in out[1 + nb:1 + nb + nq]]
        vals = np.array([float(x) for x in out[1 + nb + nq:] if x])
        o = 0
        M = vals[o:o + nb * nb].reshape(nb, nb); o += nb * nb
        S = vals[o:o + d * d * nb * nb].reshape(d, d, nb, nb); o += d * d * nb * nb
        C = vals[o:o + d * nq * nb].reshape(d, nq, nb); o += d * nq * nb
        qi = vals[o:o + nq]; o += nq
        assert o == len(vals)
        return av, aq, M, S, C, qi
    return run


def _oracle(d, k):
    """Reference tensors from the oracle's basis and quadrature (its weights
    sum to 1; scaled to the simplex volume 1/d!)."""
    lam, w = lagrange.quadrature(d, 2 * k)
    w = w / math.factorial(d)
    phi = lagrange.basis(k, d, lam)
    dl = lagrange.basis_dlam(k, d, lam)
    psi = lagrange.basis(k - 1, d, lam)
    g = [dl[:, :, a] - dl[:, :, 0] for a in range(1, d + 1)]       # d/dxi_a = d/dlam_a - d/dlam_0
    M = np.einsum("q,qi,qj->ij", w, phi, phi)
    S = np.array([[np.einsum("q,qi,qj->ij", w, g[a], g[b]) for b in range(d)] for a in range(d)])
    C = np.array([np.einsum("q,qp,qj->pj", w, psi, g[a]) for a in range(d)])
    qi = np.einsum("q,qp->p", w, psi)
    iv = [tuple(x) for x in lagrange.multi_indices(k, d)]
    iq = [tuple(x) for x in lagrange.multi_indices(k - 1, d)]
    return iv, iq, M, S, C, qi


@pytest.mark.parametrize("d,k", [(2, k) for k in range(2, 11)] + [(3, k) for k in range(2, 7)])
def test_reference_tensors_match_oracle(dump, d, k):
    av, aq, M, S, C, qi = dump(d, k)
    iv, iq, Mo, So, Co, qio = _oracle(d, k)
    pv = [iv.index(a) for a in av]         # library node -> oracle node
    pq = [iq.index(a) for a in aq]
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()   # noqa: E731
    assert rel(M, Mo[np.ix_(pv, pv)]) < 1e-13, (d, k)
    for a in range(d):
        assert rel(C[a], Co[a][np.ix_(pq, pv)]) < 1e-13, (d, k, a)
        for b in range(d):
            assert rel(S[a, b], So[a, b][np.ix_(pv, pv)]) < 1e-13, (d, k, a, b)
            assert np.array_equal(S[a, b], S[b, a].T), (d, k, a, b)   # stored exactly symmetric
    assert rel(qi, qio[pq]) < 1e-13, (d, k)
    assert abs(qi.sum() - 1 / math.factorial(d)) < 1e-14          # the pressure basis sums to one


@pytest.mark.parametrize("d,k", [(2, 2), (2, 5), (2, 10), (3, 3), (3, 6)])
def test_basis_evaluation_matches_oracle(dump, d, k):
    """RefElement::eval (the transfers evaluate the coarse basis with it) at
    seeded random points of the reference simplex and at its vertices: the
    library's Bernstein-form values equal the oracle's Silvester product to
    1e-13 relative to the largest value (both float64; at k = 10 in 2D the
    values reach about 6 and the two differ by 7.5e-14 at most)."""
    rng = np.random.default_rng(10 * d + k)
    lam = rng.dirichlet(np.ones(d + 1), size=40)
    lam = np.vstack([lam, np.eye(d + 1)])
    av, vals = dump(d, k, points=lam[:, 1:])
    iv = [tuple(x) for x in lagrange.multi_indices(k, d)]
    pv = [iv.index(a) for a in av]
    want = lagrange.basis(k, d, lam)[:, pv]
    assert vals.shape == want.shape
    assert np.abs(vals - want).max() < 1e-13 * max(1.0, np.abs(want).max()), (d, k)
