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


def test_traffic_record_matches_the_kernel_source_and_scales_by_cells():
    """The committed DRAM-traffic record is reported only for the sweep kernel
    source it was taken on (its hash covers the kernel's part of smoother.cu
    and the copy helpers); on another grid it is scaled by the cell count and
    labelled."""
    import json

    import bench

    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    at = rec["cells_captured"]
    if rec["sha256"] != bench._kernel_source_hash(rec):
        # a record taken on another kernel source is not reported
        assert bench._traffic("rbgs_f32", at) == (None, None)
        return
    got, note = bench._traffic("rbgs_f32", at)
    assert got == rec["bytes_per_sweep_full_size"] and note is None
    got8, note8 = bench._traffic("rbgs_f32", 8 * at)
    assert got8 == 8 * got and "scaled" in note8
    # traffic within a few percent of the algorithmic 16 B per node and below it
    # (the last dirty lines of u stay in L2 when the sweep ends)
    assert 0.9 * 16 * at < got <= 16 * at
