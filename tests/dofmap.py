"""Match DoFs of the CUDA library and of the oracle by position.

Both sides number DoFs their own way; a DoF is identified by (component,
node coordinates) and, for discontinuous pressure, the centroid of the
owning cell.  Coordinates of the test meshes are rationals whose
denominators divide 2^20 * 3^2 * 5 * 7, so the scaled values are integers up
to rounding error and the keys are exact."""
import numpy as np

SCALE = float(2 ** 20 * 9 * 5 * 7)


def keys(xyz, comp, center=None):
    a = np.round(np.asarray(xyz) * SCALE).astype(np.int64)
    cols = [np.asarray(comp).reshape(-1, 1).astype(np.int64), a]
    if center is not None:
        cols.append(np.round(np.asarray(center) * SCALE).astype(np.int64))
    return np.concatenate(cols, axis=1)


def permutation(k_lib, k_ora):
    """perm such that library DoF perm[i] is oracle DoF i."""
    assert k_lib.shape == k_ora.shape, (k_lib.shape, k_ora.shape)
    lib_map = {tuple(r): i for i, r in enumerate(k_lib.tolist())}
    assert len(lib_map) == len(k_lib), "duplicate library keys"
    perm = np.array([lib_map[tuple(r)] for r in k_ora.tolist()], dtype=np.int64)
    assert len(set(perm.tolist())) == len(perm)
    return perm


def oracle_free_keys(disc):
    """Keys of the oracle's free DoFs (same layout as stokes_mg_level_dofs)."""
    xyz, comp = disc.dof_coords_full()
    xyz, comp = xyz[disc.free], comp[disc.free]
    center = np.zeros_like(xyz)
    d = disc.d
    if not disc.Q.continuous:
        nV = disc.V.n
        qidx = disc.free - d * nV
        pm = qidx >= 0
        cells = np.asarray(disc.cells)
        cent = disc.verts[cells].mean(axis=1)
        owner = np.zeros(disc.Q.n, dtype=np.int64)
        for ci in range(len(cells)):
            owner[disc.Q.cell_nodes[ci]] = ci
        center[pm] = cent[owner[qidx[pm]]]
    return keys(xyz, comp, center)


def level_perm(h, level, disc):
    xyz, comp, cc = h.level_dofs(level)
    return permutation(keys(xyz, comp, cc), oracle_free_keys(disc))


def oracle_pressure_keys(disc):
    """Keys of the oracle's pressure nodes (full field order), matching
    stokes_mg_nodes' (pres_xyz, pres_cell_center)."""
    center = np.zeros_like(disc.Q.coords)
    if not disc.Q.continuous:
        cells = np.asarray(disc.cells)
        cent = disc.verts[cells].mean(axis=1)
        owner = np.zeros(disc.Q.n, dtype=np.int64)
        for ci in range(len(cells)):
            owner[disc.Q.cell_nodes[ci]] = ci
        center = cent[owner]
    return keys(disc.Q.coords, np.zeros(disc.Q.n), center)


def full_field_perms(h, disc):
    """(velocity-node perm, pressure-node perm): library node perm[i] is
    oracle node i, for the full fields of stokes_solve."""
    vx, px, pc = h.nodes()
    pv = permutation(keys(vx, np.zeros(len(vx))), keys(disc.V.coords, np.zeros(disc.V.n)))
    pq = permutation(keys(px, np.zeros(len(px)), pc), oracle_pressure_keys(disc))
    return pv, pq
