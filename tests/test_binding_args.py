"""Argument checks of the Python binding (no GPU): device vectors passed to
the library must hold at least as many elements as the C ABI reads or
writes, and outputs, which the library writes in place, must already be
contiguous float64 CUDA tensors.  Host-only handles give the sizes."""
import pytest
import torch

import workloads as W

P = pytest.importorskip("paper_2407_07253_gb300")
B = P._binding


def test_vector_checks():
    with pytest.raises(TypeError):
        B._vin([1.0, 2.0], 2, "x")
    with pytest.raises(ValueError, match="reads 5"):
        B._vin(torch.zeros(4, dtype=torch.float64), 5, "x")
    with pytest.raises(ValueError, match="float64 CUDA"):
        B._vout(torch.zeros(8, dtype=torch.float64), 8, "y")          # host tensor
    with pytest.raises(ValueError, match="float64 CUDA"):
        B._vout(torch.zeros(8, dtype=torch.float32), 8, "y")
    with pytest.raises(ValueError, match="float64 CUDA"):
        B._vout(torch.zeros(4, 4, dtype=torch.float64).t(), 16, "y")  # not contiguous
    with pytest.raises(TypeError):
        B._vout(None, 1, "y")
    assert B._rows(torch.zeros(7)) == 1 and B._rows(torch.zeros(3, 7)) == 3


def test_short_vectors_are_rejected_before_the_library_is_called():
    v, c = W.unit_square_mesh(2)
    h = P.StokesMG(v, c, 1, P.TH, 2, host_only=1)
    n = h.info()["n_free"]
    short = torch.zeros(n[0] - 1, dtype=torch.float64)
    with pytest.raises(ValueError):
        h.vcycle(short)
    with pytest.raises(ValueError):
        h.vcycle(torch.zeros(2, n[0] - 1, dtype=torch.float64))
    with pytest.raises(ValueError):
        h.fgmres(short)
    with pytest.raises(ValueError):
        h.residual(0, short, short)
    with pytest.raises(ValueError):
        h.asm(0, short)
    with pytest.raises(ValueError):
        h.arnoldi_lmax(0, short)
    with pytest.raises(ValueError):
        h.transfer(0, 0, short, torch.zeros(n[1], dtype=torch.float64))
    with pytest.raises(ValueError):
        h.coarse_solve(torch.zeros(n[-1] - 1, dtype=torch.float64))
    with pytest.raises(ValueError, match="level"):
        h.asm(len(n), torch.zeros(n[0], dtype=torch.float64))
    nv = h.info()["n_vel_nodes"] * 2
    with pytest.raises(ValueError):
        h.solve(torch.zeros(nv - 1, dtype=torch.float64))
    with pytest.raises(ValueError):
        h.solve_batched(torch.zeros(3, nv - 1, dtype=torch.float64))
    h.close()
