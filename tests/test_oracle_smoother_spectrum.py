"""The Chebyshev-ASM smoother on the spectrum of the ASM-preconditioned
Stokes operator (oracle, TH P4/P3 on the 4 x 4 square, dense eigenvalues).

M^-1 K (Eq. 3.4 with the partition of unity, Sec. 3.3) is not similar to a
symmetric matrix: its eigenvalues have imaginary parts comparable to their
real parts.  A Chebyshev residual polynomial built for a real interval
[a, b] must stay below 1 in modulus on all of them for the relaxation to
contract.  These checks pin the reason for the benchmark's relaxation
parameters: the degree-1 step contracts on both intervals tested, the
degree-2 polynomial on [0.1, 1.1] lambda_max grows above 1 off the real axis,
and on [0.5, 2.0] lambda_max it stays below 1 on every eigenvalue.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import multigrid as mg


def _spectrum(level):
    K = level.disc.K.toarray()
    n = K.shape[0]
    Minv = np.zeros((n, n))
    for p, lu in zip(level.asm.patches, level.asm.lu):
        Minv[np.ix_(p, p)] += level.asm.weight[p][:, None] * sla.lu_solve(lu, np.eye(len(p)))
    ev = np.linalg.eigvals(Minv @ K)
    return ev[np.abs(ev) > 1e-10]          # drop the constant-pressure null vector


def _residual_poly(ev, nu, lo, hi, lmax):
    """T_nu((theta - l) / delta) / T_nu(theta / delta) on [lo, hi] * lmax:
    the error factor of nu Chebyshev steps from zero (oracle.multigrid.chebyshev)."""
    a, b = lo * lmax, hi * lmax
    th, de = (a + b) / 2, (b - a) / 2
    t = lambda x: np.polynomial.chebyshev.chebval(x, [0] * nu + [1])  # noqa: E731
    return t((th - ev) / de) / t(th / de)


@pytest.fixture(scope="module")
def levels():
    v, c = W.unit_square_mesh(2)
    h = mg.Hierarchy(v, c, 1, mg.TH if hasattr(mg, "TH") else 0, [4, 2])
    return h.levels[:2]


def test_the_preconditioned_operator_has_a_complex_spectrum(levels):
    for L in levels:
        ev = _spectrum(L)
        assert np.abs(ev.imag).max() > 0.5
        assert ev.real.min() > 0            # no eigenvalue in the left half plane


def test_chebyshev_degree_one_contracts_on_both_intervals(levels):
    for L in levels:
        ev = _spectrum(L)
        for lo, hi in ((0.1, 1.1), (0.5, 2.0)):
            assert np.abs(_residual_poly(ev, 1, lo, hi, L.lmax)).max() < 1.0


def test_chebyshev_degree_two_needs_the_wide_interval(levels):
    for L in levels:
        ev = _spectrum(L)
        narrow = np.abs(_residual_poly(ev, 2, 0.1, 1.1, L.lmax))
        wide = np.abs(_residual_poly(ev, 2, 0.5, 2.0, L.lmax))
        assert narrow.max() > 1.2, narrow.max()
        # the amplified eigenvalues are the ones off the real axis
        assert np.all(np.abs(ev[narrow > 1].imag) > 0.3)
        assert wide.max() < 0.9, wide.max()
