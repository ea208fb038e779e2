"""The FBF velocity hierarchy built by the library's host code (stokes_fbf_setup
with host_only) against the oracle's (oracle/fbf.py): level sizes and the
ASMStarPC patch sets of every relaxed level, matched by node coordinates."""
import numpy as np
import pytest

import workloads as W
from oracle import fbf
from tests.dofmap import keys, permutation

P = pytest.importorskip("paper_2407_07253_gb300")


@pytest.mark.parametrize("mesh,nref,k,sched", [
    (W.unit_square_mesh(2), 1, 2, [2]),
    (W.unit_square_mesh(2), 1, 3, [3, 2]),
    (W.kuhn_cube_mesh(1), 1, 3, [3, 2]),
])
def test_velocity_levels_and_star_patches_match_oracle(mesh, nref, k, sched):
    v, c = mesh
    h = P.StokesMG(v, c, nref, P.SV, k, fbf=True, hierarchy=P.HIER_EXPLICIT, schedule=sched, host_only=1)
    st = h.info()
    vh = fbf.VelocityHierarchy(v, c, nref, sched, barycentric=True, lmax=[1.0] * 8)
    assert st["n_levels"] == len(vh.levels)
    assert list(st["n_free"][:st["n_levels"]]) == [L.disc.n_free for L in vh.levels]
    for li, L in enumerate(vh.levels[:-1]):
        off, dofs = h.patches(li)
        xyz, comp, _ = h.level_dofs(li)
        ox = L.disc.V.coords[L.disc.free]
        perm = permutation(keys(xyz, comp), keys(ox, np.zeros(len(ox))))
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        lib = {tuple(sorted(inv[dofs[off[p]:off[p + 1]]].tolist())) for p in range(len(off) - 1)}
        assert lib == {tuple(p.tolist()) for p in L.asm.patches}, li
    # the Stokes fields are the SV spaces of the finest mesh
    assert st["n_vel_nodes"] == vh.levels[0].disc.V.n
    h.close()
