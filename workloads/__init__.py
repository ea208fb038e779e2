"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only *generates inputs*: coarse meshes (vertex coordinates and
simplex connectivity), seeded nodal forcing values, per-cell viscosities and
the closed-form manufactured solution.  It holds none of the method's
arithmetic (no refinement, no finite-element spaces, no assembly, no
multigrid); both the CUDA library and the CPU oracle consume what it returns
and do everything else on their own.

The paper's benchmark problems (lid-driven cavity, backward-facing step) are
not available; the workloads below stand in for them with the same structure:
structured and unstructured simplicial meshes of the unit square, the unit
disk and the unit cube, Taylor-Hood and Scott-Vogelius pairs of order 2-4,
and nested uniform refinement (Sec. 2.1, Fig. 1; Sec. 4).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TH = 0  # Taylor-Hood P_k / P_{k-1}                           (Sec. 2.1)
SV = 1  # Scott-Vogelius P_k / P_{k-1}^disc on an Alfeld mesh (Sec. 2.1)


def unit_square_mesh(n: int):
    """Structured n x n triangulation of [0,1]^2.

    Every square is cut along the same diagonal (from its lower-right to its
    upper-left corner), so that uniform quadrisection of the n x n mesh gives
    exactly the 2n x 2n mesh of the same kind (nested hierarchy).
    Returns (verts float64 [(n+1)^2, 2], cells int32 [2 n^2, 3]).
    """
    xs = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: j * (n + 1) + i  # noqa: E731
    cells = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)
            cells.append((a, b, c))
            cells.append((b, d, c))
    return verts.astype(np.float64), np.asarray(cells, dtype=np.int32)


def kuhn_cube_mesh(n: int):
    """Structured n^3 hexahedral grid of [0,1]^3, each cube split into the
    six Kuhn (Freudenthal) tetrahedra sharing the main diagonal.
    Returns (verts float64 [(n+1)^3, 3], cells int32 [6 n^3, 4])."""
    g = np.linspace(0.0, 1.0, n + 1)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    vid = lambda i, j, k: (k * (n + 1) + j) * (n + 1) + i  # noqa: E731
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for p in perms:
                    cur = [i, j, k]
                    tet = [vid(*cur)]
                    for ax in p:
                        cur[ax] += 1
                        tet.append(vid(*cur))
                    cells.append(tet)
    return verts.astype(np.float64), np.asarray(cells, dtype=np.int32)


def delaunay_disk_mesh(seed: int = 0, h: float = 0.16, jitter: float = 0.2):
    """Seeded unstructured Delaunay triangulation of the unit disk.

    Boundary vertices are equispaced on the circle (spacing ~h); interior
    vertices sit on a square grid of spacing h (kept at distance >= 0.6 h from
    the circle) jittered by U[-jitter h, jitter h]^2 from
    numpy.random.default_rng(seed).  About 250 triangles at the default h.
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    nb = int(round(2 * math.pi / h))
    t = 2 * math.pi * np.arange(nb) / nb
    bnd = np.stack([np.cos(t), np.sin(t)], axis=1)
    g = np.arange(-1.0, 1.0 + 1e-12, h)
    X, Y = np.meshgrid(g, g, indexing="xy")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    pts = pts[np.hypot(pts[:, 0], pts[:, 1]) < 1.0 - 0.6 * h]
    pts = pts + rng.uniform(-jitter * h, jitter * h, size=pts.shape)
    verts = np.concatenate([bnd, pts], axis=0)
    tri = Delaunay(verts)
    cells = tri.simplices.astype(np.int32)
    # orient counter-clockwise and drop slivers of zero area (none expected)
    a, b, c = verts[cells[:, 0]], verts[cells[:, 1]], verts[cells[:, 2]]
    det = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = det < 0
    cells[flip] = cells[flip][:, [0, 2, 1]]
    cells = cells[np.abs(det) > 1e-12]
    return verts.astype(np.float64), cells


def nodal_forcing(n_nodes: int, dim: int, seed: int = 0) -> np.ndarray:
    """Seeded forcing f given by nodal values, U[-1, 1] per node and velocity
    component, from numpy.random.default_rng(seed).  Shape [dim, n_nodes]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(dim, n_nodes))


def cell_viscosity(n_cells: int, seed: int = 0, sigma: float = 0.5) -> np.ndarray:
    """Piecewise-constant viscosity nu_e = exp(N(0, sigma)) per cell (sigma is
    the standard deviation), from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(0.0, sigma, size=n_cells))


# --- closed-form manufactured solution on the unit square (nu = 1) ---------
def mms_velocity(x: np.ndarray) -> np.ndarray:
    """u = (sin(pi x) sin(pi y), cos(pi x) cos(pi y)); divergence-free."""
    X, Y = x[..., 0], x[..., 1]
    return np.stack([np.sin(np.pi * X) * np.sin(np.pi * Y),
                     np.cos(np.pi * X) * np.cos(np.pi * Y)], axis=-1)


def mms_pressure(x: np.ndarray) -> np.ndarray:
    """p = cos(pi x) cos(pi y); zero mean on the unit square."""
    return np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1])


def mms_forcing(x: np.ndarray) -> np.ndarray:
    """f = -Laplace(u) + grad(p) for the manufactured (u, p) above."""
    X, Y = x[..., 0], x[..., 1]
    s, c = np.sin, np.cos
    pi = np.pi
    fx = 2 * pi**2 * s(pi * X) * s(pi * Y) - pi * s(pi * X) * c(pi * Y)
    fy = 2 * pi**2 * c(pi * X) * c(pi * Y) - pi * c(pi * X) * s(pi * Y)
    return np.stack([fx, fy], axis=-1)


@dataclass
class Workload:
    """One problem: coarse mesh + refinements + discretisation + hierarchy."""
    name: str
    verts: np.ndarray
    cells: np.ndarray
    n_refine: int                 # uniform refinements of the coarse mesh
    family: int                   # TH or SV
    k: int                        # velocity degree
    schedule: list = field(default_factory=list)  # velocity degrees of the p-levels, last = hMG degree
    barycentric: bool = False     # Alfeld split of the finest mesh (SV)
    forcing: str = "nodal"        # "nodal" (seeded U[-1,1]) or "mms"
    seed: int = 0
    nu_cells: bool = False


def workload(name: str) -> Workload:
    """The synthetic problems used by the tests and the benchmark (the five
    configurations, th_p3_cube8, a small 3D case for profiling, and
    th_p4_256x256, the 2D Taylor-Hood problem at the paper's scale)."""
    if name == "th_p2_8x8":
        v, c = unit_square_mesh(2)
        return Workload(name, v, c, 2, TH, 2, [2], forcing="mms")
    if name == "th_p4_64x64":
        v, c = unit_square_mesh(8)
        return Workload(name, v, c, 3, TH, 4, [4, 2])
    if name == "th_p4_256x256":
        # the 64 x 64 problem two refinements up (about 2.7 M DoFs), the size
        # of the paper's 2D Taylor-Hood runs
        v, c = unit_square_mesh(8)
        return Workload(name, v, c, 5, TH, 4, [4, 2])
    if name == "sv_p4_disk":
        v, c = delaunay_disk_mesh(0)
        return Workload(name, v, c, 2, SV, 4, [4, 2], barycentric=True)
    if name == "th_p3_cube16":
        v, c = kuhn_cube_mesh(4)
        return Workload(name, v, c, 2, TH, 3, [3, 2])
    if name == "th_p3_cube8":
        # the 16^3 problem one refinement down: same patch structure, 1/8 of
        # the patches (a small case for profiling the batched kernels)
        v, c = kuhn_cube_mesh(4)
        return Workload(name, v, c, 1, TH, 3, [3, 2])
    if name in ("th_p6_32x32", "th_p8_32x32"):
        # high order on the 32 x 32 square; the schedule is Fig. 7's gradual
        # one (6 -> 4 -> 2, 8 -> 5 -> 2), the direct k -> 2 is the comparison
        k = int(name[4])
        v, c = unit_square_mesh(8)
        return Workload(name, v, c, 2, TH, k, [k, 4, 2] if k <= 7 else [k, 5, 2])
    if name == "th_p3_128x128_nu":
        v, c = unit_square_mesh(8)
        return Workload(name, v, c, 4, TH, 3, [3, 2], nu_cells=True)
    raise KeyError(name)
