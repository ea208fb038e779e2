"""CPU parity of the library's host-side setup (meshes, spaces, assembly of
K, transfers P / R, Vanka-star patches) against the oracle, through the
C ABI with host_only = 1 (no GPU needed).  Matrices agree entry by entry
after mapping DoFs by position; patches agree as DoF sets."""
import numpy as np
import pytest

import workloads as W
from oracle import multigrid as mg, stokes
from tests.dofmap import level_perm

P = pytest.importorskip("paper_2407_07253_gb300")

CASES = [
    # name, coarse mesh, n_refine, family, k, schedule, barycentric
    ("th_p2_8x8", W.unit_square_mesh(2), 2, 0, 2, [2], False),
    ("th_p4_8x8", W.unit_square_mesh(2), 2, 0, 4, [4, 2], False),
    ("th_p4_gradual3", W.unit_square_mesh(2), 1, 0, 4, [4, 3, 2], False),
    ("sv_p3_alfeld", W.unit_square_mesh(2), 1, 1, 3, [3, 2], True),
    ("sv_p4_disk", W.delaunay_disk_mesh(0, h=0.5), 1, 1, 4, [4, 2], True),
    ("th3d_p3", W.kuhn_cube_mesh(1), 1, 0, 3, [3, 2], False),
    ("sv3d_p3_alfeld", W.kuhn_cube_mesh(1), 0, 1, 3, [3, 2], True),
    ("th_p7_gradual", W.unit_square_mesh(2), 1, 0, 7, [7, 4, 2], False),
    ("sv_p6_gradual", W.unit_square_mesh(1), 1, 1, 6, [6, 4, 2], True),
    ("th3d_p4", W.kuhn_cube_mesh(1), 1, 0, 4, [4, 2], False),
    ("th_p10_explicit", W.unit_square_mesh(1), 1, 0, 10, [10, 9, 2], False),
]


def _build(case):
    name, (v, c), nref, fam, k, sched, bary = case
    h = P.StokesMG(v, c, nref, fam, k, barycentric=bary, host_only=1,
                   hierarchy=P.HIER_EXPLICIT, schedule=sched)
    ora = mg.Hierarchy(v, c, nref, fam, sched, barycentric=bary, lmax=[1.0] * 16)
    return h, ora


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_host_hierarchy_matches_oracle(case):
    h, ora = _build(case)
    _check_hierarchy(h, ora)


@pytest.mark.slow
def test_host_hierarchy_matches_oracle_at_bench_size():
    """The same comparison on the benchmark workload: TH P4/P3 on the 64x64
    square (167,299 free DoFs, 4225 level-0 patches), every level."""
    w = W.workload("th_p4_64x64")
    h = P.StokesMG(w.verts, w.cells, w.n_refine, w.family, w.k, barycentric=w.barycentric, host_only=1,
                   hierarchy=P.HIER_EXPLICIT, schedule=w.schedule)
    ora = mg.Hierarchy(w.verts, w.cells, w.n_refine, w.family, w.schedule, barycentric=w.barycentric,
                       lmax=[1.0] * 16)
    assert h.info()["n_free"][0] == 167299
    _check_hierarchy(h, ora)


def _check_hierarchy(h, ora):
    info = h.info()
    assert info["n_levels"] == len(ora.levels)
    perms = []
    for li, L in enumerate(ora.levels):
        assert info["n_free"][li] == L.disc.n_free
        perm = level_perm(h, li, L.disc)
        perms.append(perm)
        K = h.get_csr(li, 0)
        Kp = K[perm][:, perm]
        Ko = L.disc.K
        scale = abs(Ko).max()
        assert abs(Kp - Ko).max() <= 1e-12 * scale, (li, abs(Kp - Ko).max())
    for li, L in enumerate(ora.levels[:-1]):
        pf, pc = perms[li], perms[li + 1]
        Pm = h.get_csr(li, 1)[pf][:, pc]
        assert abs(Pm - L.P).max() <= 1e-13
        Rm = h.get_csr(li, 2)[pc][:, pf]
        assert abs(Rm - L.R).max() <= 1e-13
        off, dofs = h.patches(li)
        # each patch lists its DoFs strictly increasing (velocity components
        # blocked, then pressures): the inversion places operator entries by a
        # binary search of this list
        for i in range(len(off) - 1):
            assert np.all(np.diff(dofs[off[i]:off[i + 1]]) > 0), (li, i)
        inv = np.argsort(pf)          # library index -> oracle index
        lib_sets = sorted(tuple(sorted(inv[dofs[off[i]:off[i + 1]]].tolist())) for i in range(len(off) - 1))
        ora_sets = sorted(tuple(p.tolist()) for p in L.asm.patches)
        assert lib_sets == ora_sets


def test_host_invalid_inputs_are_rejected():
    v, c = W.unit_square_mesh(2)
    with pytest.raises(P.StokesError) as e:
        P.StokesMG(v, c, 1, 0, 1, host_only=1)                 # k < 2
    assert e.value.code == -1
    with pytest.raises(P.StokesError):
        P.StokesMG(v, c, 1, 1, 3, host_only=1)                 # SV without Alfeld
    bad = c.copy(); bad[0, 0] = 10 ** 6
    with pytest.raises(P.StokesError):
        P.StokesMG(v, bad, 1, 0, 2, host_only=1)               # vertex index out of range
    deg = c.copy(); deg[0] = [0, 0, 1]
    with pytest.raises(P.StokesError):
        P.StokesMG(v, deg, 1, 0, 2, host_only=1)               # degenerate cell
    with pytest.raises(P.StokesError):
        P.StokesMG(v, c, 0, 0, 2, host_only=1)                 # single level


def test_library_exports_every_declared_symbol():
    """Every function declared in include/stokes_mg.h is exported by the .so."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "stokes_mg.h")).read()
    names = set(re.findall(r"\b(stokes_[a-z_0-9]+)\s*\(", hdr))
    lib = P.lib()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing and len(names) >= 20, missing


_DIGEST_SCRIPT = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import workloads as W
import paper_2407_07253_gb300 as P
h = hashlib.sha256()
for v, c, nref, fam, k, sched, bary in [
        (*W.unit_square_mesh(4), 3, 0, 4, [4, 2], False),
        (*W.unit_square_mesh(2), 2, 1, 4, [4, 2], True),
        (*W.kuhn_cube_mesh(1), 2, 0, 3, [3, 2], False)]:
    m = P.StokesMG(v, c, nref, fam, k, barycentric=bary, host_only=1,
                   hierarchy=P.HIER_EXPLICIT, schedule=sched)
    for li in range(m.info()["n_levels"]):
        A = m.get_csr(li, 0)
        for a in (A.indptr, A.indices, A.data):
            h.update(np.ascontiguousarray(a).tobytes())
        if li + 1 < m.info()["n_levels"]:
            for part in (1, 2):
                T = m.get_csr(li, part)
                for a in (T.indptr, T.indices, T.data):
                    h.update(np.ascontiguousarray(a).tobytes())
            for a in m.patches(li):
                h.update(np.ascontiguousarray(a).tobytes())
print(h.hexdigest())
"""


def test_host_build_is_identical_for_any_thread_count():
    """The host build's parallel loops (atomic first-appearance numbering,
    per-thread list buffers, chunks claimed as threads come free) give the
    same numbering, operators, transfers and patches bit for bit whatever
    the number of worker threads.  The pool size is fixed per process, so
    each count runs in a child process."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    digests = {}
    for t in (1, 3, 8):
        env = dict(os.environ, STOKES_HOST_THREADS=str(t))
        out = subprocess.run([sys.executable, "-c", _DIGEST_SCRIPT, root], env=env, cwd=root,
                             capture_output=True, text=True, timeout=600)
        assert out.returncode == 0, out.stderr[-2000:]
        digests[t] = out.stdout.strip().splitlines()[-1]
    assert len(set(digests.values())) == 1, digests


def test_host_gradual_hierarchy_follows_fig7_schedule():
    """The library's GRADUAL hierarchy (no explicit schedule) takes the p-levels
    of Fig. 7 (tests/golden/pmg_schedule.txt) on the finest mesh, then the P2
    h-levels down to the coarse mesh: TH in 2D, host-only handles."""
    import os
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pmg_schedule.txt")
    rows = [l.split() for l in open(golden) if l[0] != "#"]
    v, c = W.unit_square_mesh(1)
    for k, sched in rows:
        k, sched = int(k), [int(s) for s in sched.split(",")]
        h = P.StokesMG(v, c, 2, P.TH, k, host_only=1, hierarchy=P.HIER_GRADUAL)
        info = h.info()
        nl = info["n_levels"]
        deg, mesh = info["degree"][:nl], info["mesh_index"][:nl]
        assert deg[:len(sched)] == sched and all(x == 0 for x in mesh[:len(sched)]), (k, deg, mesh)
        assert deg[len(sched) - 1:] == [2] * (nl - len(sched) + 1), (k, deg)
        assert mesh[len(sched) - 1:] == list(range(nl - len(sched) + 1)), (k, mesh)
        h.close()


def test_host_sv_hierarchy_levels():
    """Scott-Vogelius hierarchy (the reading of Sec. 3.2 / Sec. 4.2): SV P_k on the
    Alfeld-split finest mesh, the remaining Fig. 7 p-levels and the P2 level
    as Taylor-Hood on that same split mesh, then P2 h-levels on the unsplit
    finest mesh and every coarser mesh."""
    v, c = W.unit_square_mesh(1)
    for k, sched in ((3, [3, 2]), (4, [4, 2]), (6, [6, 4, 2]), (8, [8, 5, 2])):
        h = P.StokesMG(v, c, 2, P.SV, k, barycentric=True, host_only=1, hierarchy=P.HIER_GRADUAL)
        i = h.info()
        nl = i["n_levels"]
        p = len(sched)
        assert i["degree"][:nl] == sched + [2] * (nl - p), (k, i["degree"][:nl])
        assert i["level_family"][:nl] == [P.SV] + [P.TH] * (nl - 1), (k, i["level_family"][:nl])
        assert i["mesh_index"][:nl] == [0] * p + list(range(1, nl - p + 1)), (k, i["mesh_index"][:nl])
        assert i["is_p_level"][:nl] == [1] * (p - 1) + [0] * (nl - p + 1), (k, i["is_p_level"][:nl])
        assert nl - p == 3                       # meshes: split finest, finest, once refined, coarse
        h.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[3], CASES[5]], ids=[CASES[i][0] for i in (1, 3, 5)])
def test_host_hierarchy_with_cell_viscosity_matches_oracle(case):
    """A seeded per-cell viscosity on the finest cells (nu = exp(N(0, 1/4))):
    the library's K on every level, coarse cells taking their children's
    mean, equals the oracle's with the same reading.  Cells are matched by
    their centroids."""
    from oracle import geometry
    from tests.dofmap import keys, permutation
    name, (v, c), nref, fam, k, sched, bary = case
    meshes, _ = geometry.hierarchy(v, c, nref, bary)
    vf, cf = meshes[0]
    nu_o = np.exp(0.5 * np.random.default_rng(5).standard_normal(len(cf)))
    probe = P.StokesMG(v, c, nref, fam, k, barycentric=bary, host_only=1, hierarchy=P.HIER_EXPLICIT, schedule=sched)
    cent = probe.cell_centroids()
    probe.close()
    pc = permutation(keys(cent, np.zeros(len(cent))), keys(vf[cf].mean(axis=1), np.zeros(len(cf))))
    nu_l = np.empty_like(nu_o)
    nu_l[pc] = nu_o
    h = P.StokesMG(v, c, nref, fam, k, barycentric=bary, nu_cell=nu_l, host_only=1,
                   hierarchy=P.HIER_EXPLICIT, schedule=sched)
    ora = mg.Hierarchy(v, c, nref, fam, sched, barycentric=bary, nu_cells=nu_o, lmax=[1.0] * 16)
    assert h.info()["n_levels"] == len(ora.levels)
    for li, L in enumerate(ora.levels):
        perm = level_perm(h, li, L.disc)
        K = h.get_csr(li, 0)[perm][:, perm]
        assert abs(K - L.disc.K).max() <= 1e-12 * abs(L.disc.K).max(), (name, li)
    h.close()
