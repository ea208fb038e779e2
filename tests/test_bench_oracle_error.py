"""bench.py's comparison with the oracle (oracle_error), on the CPU: the
oracle's solution fed back as if the library had computed it, in the
library's node order, gives zero difference; the forcing handed to the
library is the oracle's seeded field moved to the library's nodes; and the
relaxation presets name only fields of the oracle's options."""
import os
import tempfile

import numpy as np
import pytest

import bench
import workloads as W
from oracle import multigrid as mg

P = pytest.importorskip("paper_2407_07253_gb300")


def test_relaxation_presets_are_oracle_options():
    for preset in bench.RELAX.values():
        mg.Options(**preset)


def test_oracle_error_of_the_oracle_itself_is_zero():
    w = W.workload("th_p2_8x8")
    npz = os.path.join(tempfile.mkdtemp(), "oracle.npz")
    bench.run_oracle("th_p2_8x8", "v22", save=npz)
    z = np.load(npz)
    probe = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, hierarchy=P.HIER_EXPLICIT,
                       schedule=w.schedule, host_only=1)
    vx, px, _ = probe.nodes()
    probe.close()

    def key(x):
        return [tuple(r) for r in np.round(np.asarray(x) * 1e9).astype(np.int64).tolist()]
    where_v = {k: i for i, k in enumerate(key(z["vx"]))}
    where_q = {k: i for i, k in enumerate(key(z["px"]))}
    lv = [where_v[k] for k in key(vx)]               # library node -> oracle node
    lq = [where_q[k] for k in key(px)]
    d, nV = w.verts.shape[1], len(z["vx"])
    u_o = z["full"][:d * nV].reshape(d, nV)
    p_o = z["full"][d * nV:]
    f_o = W.nodal_forcing(nV, d, w.seed)
    seen = []

    def solve(prec, f_lib, tol):
        assert np.array_equal(f_lib, f_o[:, lv])
        seen.append((prec, tol))
        ref = z["full"] if tol == bench.TOL else z["full_tight"]
        return ref[:d * nV].reshape(d, nV)[:, lv].reshape(-1), ref[d * nV:][lq]
    err = bench.oracle_error(P, W, w, npz, solve)
    assert sorted(seen) == sorted([(P.MIXED, bench.TOL), (P.FP64, bench.TOL), (P.FP64, bench.TIGHT_LIB)])
    for tag in ("mixed", "fp64", "fp64_tight"):
        assert err[tag]["u_rel"] == 0.0 and err[tag]["p_rel"] == 0.0
    # the tight solve is the discrete solution; the TOL solve is within TOL * cond of it
    assert np.abs(z["full_tight"] - z["full"]).max() < 1e-5 * np.abs(z["full"]).max()


def test_node_perm_needs_centroids_for_discontinuous_pressure():
    """Scott-Vogelius pressures are discontinuous: nodes of different cells
    share coordinates, so matching by position alone must fail loudly, and
    matching by (position, owner-cell centroid) must be a bijection."""
    xyz = np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    cen = np.array([[0.2, 0.1], [0.1, 0.2], [0.5, 0.3]])
    with pytest.raises(ValueError):
        bench.node_perm(xyz, xyz[::-1])
    perm = bench.node_perm(xyz, xyz[[2, 0, 1]], cen, cen[[2, 0, 1]])
    assert perm.tolist() == [2, 0, 1]
