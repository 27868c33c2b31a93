"""The benchmark's multi-rank bookkeeping on CPU ranks (gloo, world size 2):
the whole-job time is the slowest rank's, and the value sums the ranks'
independent solves."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # rank 1 is slower
    t = bench.max_over_ranks(ms, world, "cpu")
    out[rank] = (t, bench.whole_job_mcells(1000_000, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_with_two_gloo_ranks():
    import torch.multiprocessing as mp

    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        t, v = out[r]
        assert t == 150.0
        assert v == pytest.approx(2 * 1e6 / 0.150 / 1e6)
