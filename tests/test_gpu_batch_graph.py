"""The batched path (one launch per stage over all pairs, captured into a
CUDA graph and replayed) against the single-pair path and the oracle, and
the autotuner's choice.

Every batched kernel runs the single-pair kernel's per-point arithmetic on
its items, so a pair's results from fastncc_register_batch must equal, bit
for bit, those of sfoc_build + fastncc_match with the same correlation form
(the context's autotuned entry decides AUTO for both).  The second call of
a batch replays the graph captured by the first; the inputs are changed in
place in between, so a replay that reused stale data would fail.  A seeded
sample of points per pair is also checked against the FP64 oracle.
"""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import mixed_batch  # noqa: E402

from parity import bf16_check, bf16_oracle_side, cached, compare  # noqa: E402


@pytest.fixture(scope="module")
def b():
    import paper_2202_13347_gb300 as pkg
    pkg.build()
    return pkg.load()


@pytest.fixture(scope="module")
def ctx(b):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return b.Context(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small_batch():
    # 6 pairs at a fifth of the workload's sides and point counts: every m of
    # {41, 61, 81, 101} and R in [10, 40], ragged sizes
    return mixed_batch(seed=4100, n_pairs=6, scale=0.2)


def single_path(ctx, b, pair, p, corr):
    rc = ctx.sfoc_build(dev(pair.ref), p=p)
    sc = ctx.sfoc_build(dev(pair.sen), p=p)
    return ctx.fastncc_match(rc, sc, dev(pair.points), pair.m, pair.R, corr_path=corr)["raw"]


FORMS = {
    "f32-auto": ("f32", "auto"), "f32-direct": ("f32", "direct"), "bf16-auto": ("bf16", "auto"),
    "bf16-band": ("bf16", "band"), "bf16-column": ("bf16", "column"),
}


def corr_of(b, name):
    return {"auto": b.CORR_AUTO, "direct": b.CORR_DIRECT_F32, "band": b.CORR_TC_BAND,
            "column": b.CORR_TC_COLUMN}[name]


@pytest.mark.parametrize("form", list(FORMS))
def test_register_batch_equals_single_pair_path(b, ctx, small_batch, form):
    dt, cn = FORMS[form]
    p = b.params(dtype=b.DTYPE_BF16 if dt == "bf16" else b.DTYPE_F32)
    corr = corr_of(b, cn)
    batch = small_batch
    if cn == "column":  # the column form runs where m + 2R <= 128
        batch = [q for q in batch if q.m + 2 * q.R <= 128]
        assert batch
    refs = [dev(q.ref) for q in batch]
    sens = [dev(q.sen) for q in batch]
    pts = [dev(q.points) for q in batch]
    outs = ctx.register_batch(refs, sens, pts, [q.m for q in batch], [q.R for q in batch], p=p, corr_path=corr)
    ctx.sync()
    assert ctx.plan_count >= 1
    for q, o in zip(batch, outs):
        want = single_path(ctx, b, q, p, corr)
        ctx.sync()
        assert torch.equal(o, want), (q.m, q.R)
    ctx.release_plans()


def test_graph_replay_sees_new_inputs(b, ctx, small_batch):
    """Second call = graph replay; the images are overwritten in place (the
    reference and sensed images of each pair swapped), so the replay must
    recompute every stage from the new contents."""
    p = b.params(dtype=b.DTYPE_BF16)
    batch = small_batch
    refs = [dev(q.ref) for q in batch]
    sens = [dev(q.sen) for q in batch]
    pts = [dev(q.points) for q in batch]
    ms, Rs = [q.m for q in batch], [q.R for q in batch]
    outs = ctx.register_batch(refs, sens, pts, ms, Rs, p=p)
    first = [o.clone() for o in outs]
    plans = ctx.plan_count
    l0 = ctx.launch_count
    for i, q in enumerate(batch):  # in place: same tensors, new contents
        if q.ref.shape == q.sen.shape:
            refs[i].copy_(dev(q.sen))
            sens[i].copy_(dev(q.ref))
    ctx.register_batch(refs, sens, pts, ms, Rs, p=p, outs=outs)
    ctx.sync()
    assert ctx.plan_count == plans  # the second call replayed the first call's plan
    assert ctx.launch_count > l0
    changed = 0
    for i, q in enumerate(batch):
        swapped = type(q)(q.sen, q.ref, q.points, q.m, q.R, q.truth) if q.ref.shape == q.sen.shape else q
        want = single_path(ctx, b, swapped, p, b.CORR_AUTO)
        ctx.sync()
        assert torch.equal(outs[i], want), (q.m, q.R)
        changed += int(not torch.equal(outs[i], first[i]))
    assert changed > 0
    ctx.release_plans()


def test_register_batch_host_equals_device(b, ctx, small_batch):
    p = b.params(dtype=b.DTYPE_BF16)
    batch = small_batch[:4]
    ms, Rs = [q.m for q in batch], [q.R for q in batch]
    h_refs = [torch.from_numpy(q.ref).pin_memory() for q in batch]
    h_sens = [torch.from_numpy(q.sen).pin_memory() for q in batch]
    h_pts = [torch.from_numpy(q.points).pin_memory() for q in batch]
    for _ in range(2):  # the second call replays the plan's graph
        h_out = ctx.register_batch_host(h_refs, h_sens, h_pts, ms, Rs, p=p)
    d_out = ctx.register_batch([dev(q.ref) for q in batch], [dev(q.sen) for q in batch], [dev(q.points) for q in batch],
                               ms, Rs, p=p)
    ctx.sync()
    for h, d in zip(h_out, d_out):
        assert torch.equal(h, d.cpu())
    ctx.release_plans()


def test_register_batch_host_keeps_its_plan(b, ctx, small_batch):
    """Repeated host-buffer calls with the same buffers find the plan the
    first one built (no plan is built again; the parameters are passed as a
    fresh struct each time, so the plan key must not depend on its padding),
    and give the same results every time."""
    batch = small_batch[:4]
    ms, Rs = [q.m for q in batch], [q.R for q in batch]
    h_refs = [torch.from_numpy(q.ref).pin_memory() for q in batch]
    h_sens = [torch.from_numpy(q.sen).pin_memory() for q in batch]
    h_pts = [torch.from_numpy(q.points).pin_memory() for q in batch]
    first = ctx.register_batch_host(h_refs, h_sens, h_pts, ms, Rs, p=b.params(dtype=b.DTYPE_BF16))
    first = [o.clone() for o in first]
    built = ctx.plan_info()["plans_built"]
    for _ in range(3):
        outs = ctx.register_batch_host(h_refs, h_sens, h_pts, ms, Rs, p=b.params(dtype=b.DTYPE_BF16))
        for a, c in zip(first, outs):
            assert torch.equal(a, c)
    assert ctx.plan_info()["plans_built"] == built
    ctx.release_plans()


def _pinned_sets(batch):
    """Two input sets of the same shapes: the batch, and its images mirrored
    left to right with the points mirrored too."""
    a = ([torch.from_numpy(q.ref).pin_memory() for q in batch], [torch.from_numpy(q.sen).pin_memory() for q in batch],
         [torch.from_numpy(q.points).pin_memory() for q in batch])
    mirror = []
    for q in batch:
        pts = q.points.copy()
        pts[:, 0] = q.sen.shape[1] - 1 - pts[:, 0]
        mirror.append(pts)
    b_ = ([torch.from_numpy(np.ascontiguousarray(q.ref[:, ::-1])).pin_memory() for q in batch],
          [torch.from_numpy(np.ascontiguousarray(q.sen[:, ::-1])).pin_memory() for q in batch],
          [torch.from_numpy(np.ascontiguousarray(pt)).pin_memory() for pt in mirror])
    return a, b_


def test_submitted_batches_overlap_and_match(b, ctx, small_batch):
    """fastncc_submit_batch_host / fastncc_wait_batch_host: submissions that
    alternate between two input sets through the one staging buffer, with
    up to six outstanding (more than the four-slot event ring), each give
    the synchronous call's results for its own inputs; the plan is built
    once; an empty batch gets ticket 0; an unissued ticket is an error."""
    p = b.params(dtype=b.DTYPE_BF16)
    batch = small_batch[:4]
    ms, Rs = [q.m for q in batch], [q.R for q in batch]
    sets = _pinned_sets(batch)
    want = [[o.clone() for o in ctx.register_batch_host(*st, ms, Rs, p=p)] for st in sets]
    assert any(not torch.equal(x, y) for x, y in zip(*want))  # the two sets differ
    built = ctx.plan_info()["plans_built"]
    # two in flight at a time
    outs, tickets = [], []
    for k in range(6):
        o = [torch.empty_like(x).pin_memory() for x in want[k % 2]]
        t, o = ctx.submit_batch_host(*sets[k % 2], ms, Rs, p=p, outs=o)
        tickets.append(t)
        outs.append(o)
        if k >= 1:
            ctx.wait_batch_host(tickets[k - 1])
            assert all(torch.equal(x, y) for x, y in zip(outs[k - 1], want[(k - 1) % 2])), k - 1
    ctx.wait_batch_host(tickets[-1])
    assert all(torch.equal(x, y) for x, y in zip(outs[-1], want[1]))
    assert tickets == list(range(tickets[0], tickets[0] + 6))
    # six outstanding, then one wait for the last
    outs, tickets = [], []
    for k in range(6):
        t, o = ctx.submit_batch_host(*sets[k % 2], ms, Rs, p=p,
                                     outs=[torch.empty_like(x).pin_memory() for x in want[k % 2]])
        tickets.append(t)
        outs.append(o)
    ctx.wait_batch_host(tickets[-1])
    for k in range(6):
        assert all(torch.equal(x, y) for x, y in zip(outs[k], want[k % 2])), k
    assert ctx.plan_info()["plans_built"] == built
    # a synchronous call after submissions still matches
    again = ctx.register_batch_host(*sets[0], ms, Rs, p=p)
    assert all(torch.equal(x, y) for x, y in zip(again, want[0]))
    t0, _ = ctx.submit_batch_host([], [], [], [], [], p=p, outs=[])
    assert t0 == 0
    ctx.wait_batch_host(0)
    with pytest.raises(b.SfocError):
        ctx.wait_batch_host(tickets[-1] + 100)
    ctx.sync()
    ctx.release_plans()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_register_batch_against_oracle(b, ctx, orc, small_batch, dt):
    """A seeded sample of 6 points per pair against the FP64 oracle (BF16:
    against the oracle on its cube rounded to bf16, with the derived
    tolerances), through a graph replay."""
    p = b.params(dtype=b.DTYPE_BF16 if dt == "bf16" else b.DTYPE_F32)
    batch = small_batch
    args = ([dev(q.ref) for q in batch], [dev(q.sen) for q in batch], [dev(q.points) for q in batch],
            [q.m for q in batch], [q.R for q in batch])
    outs = ctx.register_batch(*args, p=p)
    outs = ctx.register_batch(*args, p=p, outs=outs)  # replay
    ctx.sync()
    for k, q in enumerate(batch):
        rng = np.random.default_rng(700 + k)
        idx = np.sort(rng.choice(len(q.points), min(6, len(q.points)), replace=False))
        sub = type(q)(q.ref, q.sen, q.points[idx], q.m, q.R, q.truth[idx])
        g = {key: v[torch.from_numpy(idx).cuda()] for key, v in b.results(outs[k]).items()}
        if dt == "f32":
            o = cached(("graph-f32", k), lambda: orc.match_pair(sub.ref, sub.sen, sub.points, sub.m, sub.R,
                                                                want_maps=True))
            compare(g, o, q.R, oracle_maps=o["maps"])
        else:
            o_r, o_u, regions = cached(("graph-bf16", k), lambda: bf16_oracle_side(orc, sub, roi=True))
            bf16_check(g, o_r, o_u, regions, q.R, {})
    ctx.release_plans()


@pytest.mark.parametrize("dt", ["f32", "bf16"])
def test_autotuner_keeps_the_fastest_measured_form(b, ctx, small_batch, dt):
    """After an AUTO match the context holds an entry for (dtype, m, R) whose
    choice is the candidate with the shortest measured time; the entry
    survives an export / import round trip into another context."""
    p = b.params(dtype=b.DTYPE_BF16 if dt == "bf16" else b.DTYPE_F32)
    q = small_batch[0]
    single_path(ctx, b, q, p, b.CORR_AUTO)
    ctx.sync()
    e = ctx.autotune_entry(p.cube_dtype, q.m, q.R)
    assert e is not None and e["sample"] > 0 and len(e["candidates"]) >= 2
    timed = [c for c in e["candidates"] if c[2] >= 0]
    best = min(timed, key=lambda c: c[2])
    assert (e["path"], e["option"]) == (best[0], best[1])
    text = ctx.autotune_export()
    rec = json.loads(text)
    assert any(r["m"] == q.m and r["R"] == q.R and r["path"] == e["path"] for r in rec["entries"])
    other = b.Context(0)
    assert other.autotune_entry(p.cube_dtype, q.m, q.R) is None
    other.autotune_import(text)
    assert other.autotune_entry(p.cube_dtype, q.m, q.R)["path"] == e["path"]
    with pytest.raises(b.SfocError):
        other.autotune_import('{"entries": [{"dtype": 0, "m": 101, "R": 40, "path": 6, "option": 128, '
                              '"candidates": []}]}')  # the Fourier form does not run for m + 2R = 181
    other.close()


def test_match_and_build_batch_replay(b, ctx, small_batch):
    """sfoc_build_batch and fastncc_match_batch keep plans too: a repeated
    call replays them and gives the same results."""
    p = b.params(dtype=b.DTYPE_F32)
    batch = small_batch
    imgs = [dev(q.ref) for q in batch] + [dev(q.sen) for q in batch]
    cubes = ctx.sfoc_build_batch(imgs, p=p)
    n = len(batch)
    args = (cubes[:n], cubes[n:], [dev(q.points) for q in batch], [q.m for q in batch], [q.R for q in batch])
    o1 = ctx.fastncc_match_batch(*args)
    ctx.sync()
    first = [o.clone() for o in o1]
    plans = ctx.plan_count
    for o in o1:
        o.zero_()
    cubes2 = ctx.sfoc_build_batch(imgs, p=p, outs=cubes)  # replayed build into the same cubes
    assert all(c2 is c for c2, c in zip(cubes2, cubes))
    o2 = ctx.fastncc_match_batch(*args, outs=o1)
    ctx.sync()
    assert ctx.plan_count == plans  # both calls found their plans
    for a, c in zip(first, o2):
        assert torch.equal(a, c)
    ctx.release_plans()
