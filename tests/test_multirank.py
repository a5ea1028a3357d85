"""The bench's multi-rank bookkeeping on CPU with two gloo ranks: each replica's
times are reduced to the slowest one on every rank, the whole-job value counts
every replica's work over that time, and the reference arm does its work on
rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        a4, step = bench.aggregate_times(100.0 + 50.0 * rank, 1000.0 - 10.0 * rank, world, "cpu")
        dist.barrier()
        ref = bench.run_reference(None, rank, world) if rank != 0 else "rank0"
        q.put((rank, a4, step, bench.job_tflops(world, 1.6e14, a4), ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, a4, step, val, ref in out:
        assert a4 == 150.0 and step == 1000.0
        assert val == pytest.approx(2 * 1.6e14 / 0.150 / 1e12)
    assert out[1][4] is None  # rank 1 of the reference arm returns without work


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_times(12.5, 40.0, 1, "cpu") == (12.5, 40.0)
    assert bench.job_tflops(1, 1e12, 1000.0) == pytest.approx(1.0)
