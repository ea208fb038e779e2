"""The allocation-free batched inverse (stokes_batched_inverse_noalloc) for
callers that cannot allocate device memory, checked through the C ABI
against the allocating entry point stokes_mg_patch_inverses on the same
patch matrices, on two calls in a row.

The case (Taylor-Hood P3/P2 on a 4^3 Kuhn mesh) has patches of 20 to 540
DoFs, so both the shared-memory kernel and the global-memory kernel (whose
pivot workspace lives in the library's fixed scratch array) run.  This file
is collected last on purpose."""
import ctypes
from ctypes import byref, c_int, c_void_p

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
P = pytest.importorskip("paper_2407_07253_gb300")

pytestmark = pytest.mark.gpu

TOL = 1e-10   # the tolerance of the patch-inverse parity test (cond * eps)


def _call(sizes, mats):
    first = c_int(-2)
    stream = c_void_p(torch.cuda.current_stream().cuda_stream)
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
