"""Multi-rank logic of bench.py on CPU: two gloo ranks.

Each rank times its own replica (weak scaling); the job's figures are the
slowest rank's time and the sum of the points matched by all ranks, and
every rank draws its own seeded pair.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, ms, matched, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.reduce_over_ranks(dist, torch, ms[rank], matched[rank], "cpu")
        p, _ = bench.workload("inverting512", rank)
        q.put((rank, got, float(p.ref[0, :8].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_sum_points():
    world = 2
    ms, matched = [10.5, 12.25], [900, 950]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ms, matched, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, got, _ in out:
        assert got == (12.25, 1850)
    # each rank draws its own pair
    assert out[0][2] != out[1][2]


def test_single_rank_and_job_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, torch, 7.0, 5, "cpu") == (7.0, 5)
    # 1850 points per step, 10 steps in 20 ms -> 925000 CP/s
    assert bench.job_value(1850, 10, 20.0) == pytest.approx(925000.0)
