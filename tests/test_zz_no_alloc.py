"""The allocation-free batched inverse (stokes_batched_inverse_noalloc) for
callers that cannot allocate device memory, checked through the C ABI
against the allocating entry point stokes_mg_patch_inverses on the same
patch matrices, on two calls in a row.

The case (Taylor-Hood P3/P2 on a 4^3 Kuhn mesh) has patches of 20 to 540
DoFs, so both the shared-memory kernel and the global-memory kernel (whose
pivot workspace lives in the library's fixed scratch array) run.  This file
is collected last on purpose."""
import ctypes
import threading
from ctypes import byref, c_int, c_void_p

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the tolerance of the patch-inverse parity test (cond * eps)


def _call(sizes, mats, stream=None):
    first = c_int(-2)
    stream = c_void_p((stream or torch.cuda.current_stream()).cuda_stream)
    rc = P.lib().stokes_batched_inverse_noalloc(len(sizes), sizes.ctypes.data_as(c_void_p),
                                                c_void_p(mats.data_ptr()), byref(first), stream)
    return rc, first.value


def test_noalloc_inverse_matches_allocating_entry_point():
    v, c = W.kuhn_cube_mesh(2)
    h = P.StokesMG(v, c, 1, 0, 3, hierarchy=P.HIER_EXPLICIT, schedule=[3, 2])
    off, _ = h.patches(0)
    sizes = np.ascontiguousarray(np.diff(off), dtype=np.int32)
    assert sizes.min() <= 160 < sizes.max()
    K = h.patch_matrices(0)          # gathered patch matrices, row-major
    ref = h.patch_inverses(0)        # allocating entry point
    h.close()
    first_result = None
    for call in range(2):
        mats = torch.tensor(K, device="cuda")
        rc, fs = _call(sizes, mats)
        assert rc == 0, P.lib().stokes_noalloc_last_error().decode()
        assert fs == -1
        got = mats.cpu().numpy()
        pos = 0
        for n in sizes:
            a = got[pos:pos + n * n]
            b = ref[pos:pos + n * n]
            assert np.abs(a - b).max() <= TOL * np.abs(b).max()
            pos += n * n
        if first_result is None:
            first_result = got
        else:
            assert np.array_equal(got, first_result)


def test_noalloc_rejects_oversized_and_reports_singular():
    big = np.full(2000, 300, dtype=np.int32)                 # sum 600000 > limit
    mats = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc, _ = _call(big, mats)
    assert rc == -1 and b"exceeds" in P.lib().stokes_noalloc_last_error()
    rc, _ = _call(np.zeros(0, dtype=np.int32), mats)
    assert rc == -1
    sizes = np.array([3, 2], dtype=np.int32)
    m = torch.tensor(np.concatenate([np.eye(3).ravel(), np.zeros(4)]), device="cuda")
    rc, fs = _call(sizes, m)
    assert rc == -3 and fs == 1
    assert torch.equal(m[:9].cpu(), torch.eye(3, dtype=torch.float64).reshape(-1))


def test_noalloc_concurrent_host_threads():
    """Two host threads call the entry point at the same time, each on its
    own stream with its own patch sizes and matrices (ctypes releases the
    interpreter lock during the call).  The calls share the static host
    staging arrays and the device scratch; the entry point serialises them,
    so every result is still the inverse of that thread's own matrices."""
    v, c = W.kuhn_cube_mesh(2)
    h = P.StokesMG(v, c, 1, 0, 3, hierarchy=P.HIER_EXPLICIT, schedule=[3, 2])
    off, _ = h.patches(0)
    sizes = np.ascontiguousarray(np.diff(off), dtype=np.int32)
    K = h.patch_matrices(0)
    ref = h.patch_inverses(0)
    h.close()
    # thread 0: every patch of the level; thread 1: the first half of the
    # patches, scaled by 2 (its inverses are the references halved)
    half = len(sizes) // 2
    n_half = int((sizes[:half].astype(np.int64) ** 2).sum())
    jobs = [(sizes, K, ref), (np.ascontiguousarray(sizes[:half]), 2.0 * K[:n_half], 0.5 * ref[:n_half])]
    errors = [None, None]

    def work(t):
        sz, mat, want = jobs[t]
        st = torch.cuda.Stream()
        try:
            for _ in range(3):
                with torch.cuda.stream(st):
                    m = torch.tensor(mat, device="cuda")
                st.synchronize()
                rc, fs = _call(sz, m, st)
                assert rc == 0 and fs == -1, (rc, fs)
                got = m.cpu().numpy()
                pos = 0
                for n in sz:
                    a, b = got[pos:pos + n * n], want[pos:pos + n * n]
                    assert np.abs(a - b).max() <= TOL * np.abs(b).max()
                    pos += n * n
        except Exception as e:  # noqa: BLE001
            errors[t] = e

    th = [threading.Thread(target=work, args=(t,)) for t in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert errors == [None, None], errors
