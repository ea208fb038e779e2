"""Host logic of the multi-GPU bench path (replicas only: each rank runs the
whole step on its own GPU; the ranks only agree on the slowest step time).
Runs as two gloo processes on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    v = bench.max_over_ranks(10.0 + 3.5 * rank, dist, torch.device("cpu"))
    dist.barrier()
    out[rank] = (r, w, local, v)
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_replicas():
    world = 2
    port = _free_port()
    # spawn, not fork: the test process may already run the library's host threads
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, local, v) in res.items():
        assert (r, w, local) == (rank, world, rank)
        assert v == 13.5          # the slowest replica's time on every rank


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(7.25, None, None) == 7.25
