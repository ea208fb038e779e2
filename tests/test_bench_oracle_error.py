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

    def solve(prec, f_lib):
        assert np.array_equal(f_lib, f_o[:, lv])
        seen.append(prec)
        return u_o[:, lv].reshape(-1), p_o[lq]
    err = bench.oracle_error(P, W, w, npz, solve)
    assert sorted(seen) == sorted([P.MIXED, P.FP64])
    for tag in ("mixed", "fp64"):
        assert err[tag]["u_rel"] == 0.0 and err[tag]["p_rel"] == 0.0
