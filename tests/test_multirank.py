"""Multi-rank paths on CPU with two gloo ranks: the bench's bookkeeping (each
replica's times are reduced to the slowest one on every rank, the whole-job
value counts every replica's work over that time, the reference arm works on
rank 0 only) and the outer-grid partition of a sharded W build (each rank's
partial kernel over its slice, summed by one all-reduce, is the full W)."""
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


def _shard_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import numpy as np
    import torch
    import torch.distributed as dist
    from synth import workloads as wl
    from oracle import wbuild
    from paper_2607_17314_b300.api import grid_shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = wl.tiny_chain(n_atom=2, n_rad=9, n_ang=14, shells=(0, 1), n_mu=13, seed=21)
        xi = wl.seeded_matrix((13, w.n_g), 31, 1e-2)
        xit = wl.seeded_matrix((3, 13, w.n_g), 32, 1e-2)
        g0, g1 = grid_shard(w.n_g, rank, world)
        rows = np.arange(g0, g1)
        calG = wbuild.stage1(w.grid_xyz, w.grid_w, xi, w.jastrow, g_rows=rows)
        part = torch.as_tensor(wbuild.stage2(w.grid_w, xi, xit, calG, g_rows=rows))
        dist.all_reduce(part)                       # the one exchange step
        full, _ = wbuild.build(w.grid_xyz, w.grid_w, xi, xit, w.jastrow)
        err = float(np.max(np.abs(part.numpy() - full)) / np.max(np.abs(full)))
        q.put((rank, g0, g1, w.n_g, err))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_w_equals_full_w():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, a0, a1, n_g, e0), (_, b0, b1, _, e1) = out
    assert (a0, a1, b0, b1) == (0, a1, a1, n_g) and 0 < a1 < n_g and a1 % 64 == 0
    assert e0 < 1e-13 and e1 < 1e-13


def test_grid_shard_partition():
    sys.path.insert(0, ROOT)
    from paper_2607_17314_b300.api import grid_shard
    for n_g in (1, 63, 64, 65, 1000, 100000):
        for world in (1, 2, 3, 8):
            sl = [grid_shard(n_g, r, world) for r in range(world)]
            assert sl[0][0] == 0 and sl[-1][1] == n_g
            assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
            assert all(g0 % 64 == 0 for g0, _ in sl)
            sizes = [g1 - g0 for g0, g1 in sl]
            assert max(sizes) - min(sizes) <= 64
