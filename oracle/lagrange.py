"""Equispaced Lagrange P_k on a d-simplex and quadrature.  Oracle: test
infrastructure.

The paper uses continuous P_k velocity with continuous (Taylor-Hood) or
discontinuous (Scott-Vogelius) P_{k-1} pressure (Sec. 2.1).  It does not fix
the nodal basis; this oracle reads it as the equispaced lattice, whose nodes
are the points sum_i (alpha_i / k) v_i for multi-indices |alpha| = k over the
d+1 vertices.  The basis is Silvester's closed form in barycentric
coordinates

    phi_alpha(lambda) = prod_i prod_{j < alpha_i} (k lambda_i - j) / (j + 1),

which is 1 at its own node and 0 at every other lattice node.
"""
from functools import lru_cache
from itertools import product

import numpy as np
from scipy.special import roots_jacobi


@lru_cache(maxsize=None)
def multi_indices(k: int, d: int):
    """All alpha in N^{d+1} with |alpha| = k, in decreasing lexicographic
    order (so that for k = 1 local node i is vertex i)."""
    out = [a for a in product(range(k + 1), repeat=d + 1) if sum(a) == k]
    return tuple(sorted(out, reverse=True))


def _s(m, k, t):
    """s_m(t) = prod_{j<m} (k t - j)/(j+1)."""
    r = np.ones_like(t)
    for j in range(m):
        r = r * (k * t - j) / (j + 1)
    return r


def _ds(m, k, t):
    """d/dt s_m(t) by the product rule."""
    r = np.zeros_like(t)
    for l in range(m):
        term = np.full_like(t, k / (l + 1))
        for j in range(m):
            if j != l:
                term = term * (k * t - j) / (j + 1)
        r = r + term
    return r


def basis(k: int, d: int, lam: np.ndarray) -> np.ndarray:
    """Values phi_alpha at barycentric points lam [..., d+1] -> [..., nb]."""
    if k == 0:
        return np.ones(lam.shape[:-1] + (1,))
    cols = []
    for a in multi_indices(k, d):
        v = np.ones(lam.shape[:-1])
        for i in range(d + 1):
            v = v * _s(a[i], k, lam[..., i])
        cols.append(v)
    return np.stack(cols, axis=-1)


def basis_dlam(k: int, d: int, lam: np.ndarray) -> np.ndarray:
    """Derivatives d phi_alpha / d lambda_i treating the lambda_i as
    independent variables -> [..., nb, d+1].  The physical gradient is
    sum_i (d phi / d lambda_i) grad(lambda_i)."""
    if k == 0:
        return np.zeros(lam.shape[:-1] + (1, d + 1))
    out = []
    for a in multi_indices(k, d):
        row = []
        for i in range(d + 1):
            v = _ds(a[i], k, lam[..., i])
            for m in range(d + 1):
                if m != i:
                    v = v * _s(a[m], k, lam[..., m])
            row.append(v)
        out.append(np.stack(row, axis=-1))
    return np.stack(out, axis=-2)


def quadrature(d: int, degree: int):
    """Stroud conical-product rule on the reference simplex, exact for total
    degree `degree`.  Returns (barycentric points [nq, d+1], weights [nq])
    with weights summing to 1 (multiply by |T|).

    Collapsed coordinates: 2D  x = a, y = b (1-a), Jacobian (1-a);
                           3D  x = a, y = b (1-a), z = c (1-a)(1-b),
                               Jacobian (1-a)^2 (1-b).
    The Jacobian powers are absorbed by Gauss-Jacobi weights (1-t)^alpha.
    """
    n = degree // 2 + 1

    def gj(alpha):
        t, w = roots_jacobi(n, alpha, 0.0)
        # map [-1,1] -> [0,1]; (1-t)^alpha = 2^alpha (1-x)^alpha, dt = 2 dx
        return (t + 1.0) / 2.0, w / 2.0 ** (alpha + 1)

    if d == 2:
        a, wa = gj(1.0)
        b, wb = gj(0.0)
        A, B = np.meshgrid(a, b, indexing="ij")
        W = np.outer(wa, wb)
        x = A
        y = B * (1 - A)
        pts = np.stack([1 - x - y, x, y], axis=-1).reshape(-1, 3)
        w = W.reshape(-1) / 0.5
    elif d == 3:
        a, wa = gj(2.0)
        b, wb = gj(1.0)
        c, wc = gj(0.0)
        A, B, C = np.meshgrid(a, b, c, indexing="ij")
        W = wa[:, None, None] * wb[None, :, None] * wc[None, None, :]
        x = A
        y = B * (1 - A)
        z = C * (1 - A) * (1 - B)
        pts = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
        w = W.reshape(-1) / (1.0 / 6.0)
    else:
        raise ValueError(d)
    return pts, w


def barycentric_gradients(verts, cells):
    """grad(lambda_i) per cell -> [nc, d+1, d], and the cell volumes."""
    cells = np.asarray(cells)
    d = cells.shape[1] - 1
    J = np.stack([verts[cells[:, i + 1]] - verts[cells[:, 0]] for i in range(d)], axis=2)
    Jinv = np.linalg.inv(J)                 # rows: grad(lambda_1..d)
    g0 = -Jinv.sum(axis=1, keepdims=True)   # grad(lambda_0)
    G = np.concatenate([g0, Jinv], axis=1)
    fact = 2.0 if d == 2 else 6.0
    vol = np.abs(np.linalg.det(J)) / fact
    return G, vol


def to_barycentric(verts, cell, x):
    """Barycentric coordinates of points x [m, d] in the simplex `cell`."""
    v = verts[np.asarray(cell)]
    d = v.shape[1]
    J = (v[1:] - v[0]).T
    lam_rest = np.linalg.solve(J, (np.asarray(x) - v[0]).T).T
    return np.concatenate([1 - lam_rest.sum(axis=1, keepdims=True), lam_rest], axis=1)
