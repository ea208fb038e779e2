"""Simplicial meshes: uniform refinement R_u, barycentric (Alfeld) refinement
R_b, boundary entities (Sec. 2.1, Fig. 1; Sec. 3.3 on nested hierarchies with
barycentric refinement of the finest mesh only).  Oracle: test infrastructure.

A mesh is a pair (verts [nv, d] float64, cells [nc, d+1] int).  Refinements
also return ``parent`` [nc_fine] = index of the coarse cell that contains each
fine cell, which the h-transfer needs.
"""
from itertools import combinations

import numpy as np


def _midpoint_table(verts, cells):
    """Map each edge (sorted vertex pair) to a new midpoint vertex index."""
    d = cells.shape[1] - 1
    edges = {}
    new = [v for v in verts]
    nv = len(verts)
    for c in cells:
        for a, b in combinations(c.tolist(), 2):
            key = (min(a, b), max(a, b))
            if key not in edges:
                edges[key] = nv
                new.append(0.5 * (verts[a] + verts[b]))
                nv += 1
    return np.asarray(new, dtype=np.float64), edges


def refine_uniform(verts, cells):
    """One step of uniform refinement R_u (Fig. 1 middle).

    2D: quadrisection of each triangle into 3 corner triangles and the middle
    one.  3D: Bey's regular refinement of each tetrahedron into 4 corner
    tetrahedra and 4 from the inner octahedron cut along the x02-x13 diagonal.
    """
    cells = np.asarray(cells)
    d = cells.shape[1] - 1
    nverts, edges = _midpoint_table(verts, cells)
    m = lambda a, b: edges[(min(a, b), max(a, b))]  # noqa: E731
    out, parent = [], []
    for ci, c in enumerate(cells.tolist()):
        if d == 2:
            a, b, cc = c
            ab, bc, ca = m(a, b), m(b, cc), m(cc, a)
            kids = [(a, ab, ca), (ab, b, bc), (ca, bc, cc), (ab, bc, ca)]
        else:
            x0, x1, x2, x3 = c
            x01, x02, x03 = m(x0, x1), m(x0, x2), m(x0, x3)
            x12, x13, x23 = m(x1, x2), m(x1, x3), m(x2, x3)
            kids = [(x0, x01, x02, x03), (x01, x1, x12, x13),
                    (x02, x12, x2, x23), (x03, x13, x23, x3),
                    (x01, x02, x03, x13), (x01, x02, x12, x13),
                    (x02, x03, x13, x23), (x02, x12, x13, x23)]
        out.extend(kids)
        parent.extend([ci] * len(kids))
    return nverts, np.asarray(out, dtype=np.int64), np.asarray(parent, dtype=np.int64)


def refine_alfeld(verts, cells):
    """Barycentric refinement R_b with the Alfeld split (Fig. 1 right): each
    simplex is split into d+1 simplices joining its barycenter to its facets."""
    cells = np.asarray(cells)
    d = cells.shape[1] - 1
    new = [v for v in verts]
    nv = len(verts)
    out, parent = [], []
    for ci, c in enumerate(cells.tolist()):
        g = np.mean(verts[c], axis=0)
        new.append(g)
        gi = nv
        nv += 1
        for drop in range(d + 1):
            facet = [c[i] for i in range(d + 1) if i != drop]
            # keep orientation: replace the dropped vertex by the barycenter
            kid = list(c)
            kid[drop] = gi
            out.append(tuple(kid))
            parent.append(ci)
    return np.asarray(new, dtype=np.float64), np.asarray(out, dtype=np.int64), np.asarray(parent, dtype=np.int64)


def boundary_entities(cells):
    """All vertex subsets (entities of every dimension < d) that lie on the
    boundary, i.e. that are contained in a facet owned by exactly one cell."""
    cells = np.asarray(cells)
    d = cells.shape[1] - 1
    count = {}
    for c in cells.tolist():
        for f in combinations(sorted(c), d):
            count[f] = count.get(f, 0) + 1
    bnd = set()
    for f, n in count.items():
        if n == 1:
            for r in range(1, d + 1):
                for sub in combinations(f, r):
                    bnd.add(sub)
    return bnd


def cell_volumes(verts, cells):
    """|T| = |det(v1-v0, ..., vd-v0)| / d!"""
    cells = np.asarray(cells)
    d = cells.shape[1] - 1
    J = np.stack([verts[cells[:, i + 1]] - verts[cells[:, 0]] for i in range(d)], axis=2)
    fact = 1.0
    for i in range(2, d + 1):
        fact *= i
    return np.abs(np.linalg.det(J)) / fact


def hierarchy(verts, cells, n_refine, barycentric=False):
    """Nested meshes [M_0 (finest), M_1, ..., M_L (coarsest)] with the parent
    map of every mesh into the next coarser one (Sec. 3.1: standard coarsening
    doubles h per level; Sec. 3.3: barycentric refinement only on the finest)."""
    meshes = [(np.asarray(verts, dtype=np.float64), np.asarray(cells, dtype=np.int64))]
    parents = []
    for _ in range(n_refine):
        v, c, p = refine_uniform(*meshes[-1])
        meshes.append((v, c))
        parents.append(p)
    if barycentric:
        v, c, p = refine_alfeld(*meshes[-1])
        meshes.append((v, c))
        parents.append(p)
    meshes = meshes[::-1]
    parents = parents[::-1]   # parents[i] maps cells of meshes[i] into meshes[i+1]
    return meshes, parents
