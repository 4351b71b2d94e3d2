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


# ---- sharding one job over ranks (pairs, or row bands of one pair) ----------

def _oracle_rows(o):
    """The oracle's per-point results as (n, 6) rows like the library's."""
    import numpy as np
    return np.stack([o["dx"], o["dy"], o["ncc"], o["sub_dx"], o["sub_dy"], o["status"]], 1).astype(np.float64)


def _shard_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    from paper_2202_13347_gb300 import shard
    from workloads import tiny_pair
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # (1) by pairs: three small pairs, balanced over the ranks by cost
        pairs = [tiny_pair(60 + i, 70 + 9 * i, 80, 11 + 2 * i, 3 + i, 5, shift=(1, -2)) for i in range(3)]
        costs = [shard.pair_cost(len(q_.points), q_.m, q_.R, q_.ref.size) for q_ in pairs]
        mine = shard.shard_pairs(costs, world)[rank]
        offs = np.cumsum([0] + [len(q_.points) for q_ in pairs])
        idx, rows = [], []
        for i in mine:
            q_ = pairs[i]
            o = oracle.match_pair(q_.ref, q_.sen, q_.points, q_.m, q_.R, roi=False)
            idx.append(np.arange(offs[i], offs[i + 1]))
            rows.append(_oracle_rows(o))
        by_pairs = shard.gather_results(dist, rank, world, int(offs[-1]),
                                        np.concatenate(idx) if idx else np.zeros(0, np.int64),
                                        np.concatenate(rows) if rows else np.zeros((0, 6)))
        # (2) by row bands of one tall pair: each rank builds the cube of its
        # slice only (whole-slice SFOC, borders clamped at the slice's edges)
        big = tiny_pair(77, 230, 90, 15, 4, 24, shift=(2, 1))
        bands = shard.row_bands(big.ref.shape[0], big.sen.shape[0], big.points, big.m, big.R, world)
        b = bands[rank]
        r_s, s_s, pts = shard.band_inputs(big.ref, big.sen, big.points, b)
        o = oracle.match_pair(r_s, s_s, pts, big.m, big.R, roi=False)
        by_rows = shard.gather_results(dist, rank, world, len(big.points), b.points, _oracle_rows(o))
        q.put((rank, by_pairs, by_rows, [len(x.points) for x in bands]))
    finally:
        dist.destroy_process_group()


def test_sharded_job_gathers_the_single_rank_results():
    """Two gloo ranks split one job (by pairs, and one pair by row bands with
    the SFOC halo), match their shards with the oracle as the stand-in for
    the library, and gather the results to rank 0: exactly the single-rank
    results, every point once, in the original order."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from workloads import tiny_pair
    oracle.build()
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted([q.get(timeout=400) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, by_pairs, by_rows, band_sizes = out[0]
    assert out[1][1] is None and out[1][2] is None  # only rank 0 holds the gathered job
    assert all(n > 0 for n in band_sizes)            # both bands have points
    pairs = [tiny_pair(60 + i, 70 + 9 * i, 80, 11 + 2 * i, 3 + i, 5, shift=(1, -2)) for i in range(3)]
    want = np.concatenate([_oracle_rows(oracle.match_pair(q_.ref, q_.sen, q_.points, q_.m, q_.R, roi=False))
                           for q_ in pairs])
    np.testing.assert_array_equal(by_pairs, want)
    big = tiny_pair(77, 230, 90, 15, 4, 24, shift=(2, 1))
    want = _oracle_rows(oracle.match_pair(big.ref, big.sen, big.points, big.m, big.R, roi=False))
    np.testing.assert_array_equal(by_rows, want)


def test_shard_rules():
    sys.path.insert(0, ROOT)
    import numpy as np
    from paper_2202_13347_gb300 import shard
    # LPT: every pair once, loads within the largest single cost of each other
    costs = [9.0, 7.0, 6.0, 5.0, 4.0, 1.0]
    parts = shard.shard_pairs(costs, 2)
    assert sorted(sum(parts, [])) == list(range(6))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(costs)
    # bands: every point once; a band's slice covers every row its points read plus the halo
    pts = np.array([[40, y] for y in range(30, 200, 7)], np.int32)
    bands = shard.row_bands(230, 230, pts, 15, 4, 3)
    assert sorted(np.concatenate([b.points for b in bands]).tolist()) == list(range(len(pts)))
    h = shard.template_half(15)
    for b in bands:
        for k in b.points:
            y = pts[k, 1]
            assert b.s0 <= max(0, y - h - 4 - shard.HALO) and b.s1_ref >= min(230, y - h + 15 + 4 + shard.HALO)
