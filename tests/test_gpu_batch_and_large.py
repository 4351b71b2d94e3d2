"""The mixed batch of pairs and the 10000^2 pair against the oracle.

Mixed batch: pairs of different sizes, radiometric maps, m in {41, 61, 81, 101} and
R in [10, 40], built and matched through the batched entry points
(sfoc_build_batch, fastncc_match_batch), F32 and BF16 forms; the oracle
checks a seeded sample of points per pair.
10000^2 pair: at full size, the 16-bit reference read through
sfoc_build_u16; 10000 points, m = 101, R = 40 (the BF16 form takes the
band tensor-core kernel: m + 2R = 181 rules the column form out, and the
band form issues fewer MMAs than the Toeplitz one); the oracle checks a seeded
sample of points.  Tolerances as in the other parity tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import mixed_batch, speckle_pair_10000  # noqa: E402

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


def sample(pair, k, seed):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pair.points), min(k, len(pair.points)), replace=False))
    return idx, type(pair)(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R, pair.truth[idx])


@pytest.fixture(scope="module")
def batch():
    # 16 of the 64 pairs at a quarter of the side lengths and point counts
    return mixed_batch(n_pairs=16, scale=0.25)


PER_PAIR = 8  # oracle points per pair of the mixed batch


def oracle_f32(orc, batch, k):
    pair = batch[k]
    idx, sub = sample(pair, PER_PAIR, 400 + k)
    o = cached(("mixed-f32", k), lambda: orc.match_pair(sub.ref, sub.sen, sub.points, sub.m, sub.R, want_maps=True))
    return idx, o


@pytest.mark.parametrize("path", ["direct", "auto"])
def test_mixed_batch_f32(b, ctx, orc, batch, path):
    """F32 cubes: the plain direct correlation, and the automatic choice
    (the Fourier correlation of Eq. 13 wherever m + 2R <= 128, so it runs on
    the batch's ragged m and R)."""
    corr = {"direct": b.CORR_DIRECT_F32, "auto": b.CORR_AUTO}[path]
    refs = ctx.sfoc_build_batch([dev(p.ref) for p in batch])
    sens = ctx.sfoc_build_batch([dev(p.sen) for p in batch])
    outs = ctx.fastncc_match_batch(refs, sens, [dev(p.points) for p in batch], [p.m for p in batch], [p.R for p in batch],
                                   corr_path=corr)
    ctx.sync()
    for k, pair in enumerate(batch):
        g = b.results(outs[k])
        idx, o = oracle_f32(orc, batch, k)
        gi = {key: v[torch.from_numpy(idx).cuda()] for key, v in g.items()}
        compare(gi, o, pair.R, oracle_maps=o["maps"])


def test_mixed_batch_bf16(b, ctx, orc, batch):
    p = b.params(dtype=b.DTYPE_BF16)
    refs = ctx.sfoc_build_batch([dev(pp.ref) for pp in batch], p=p)
    sens = ctx.sfoc_build_batch([dev(pp.sen) for pp in batch], p=p)
    outs = ctx.fastncc_match_batch(refs, sens, [dev(pp.points) for pp in batch], [pp.m for pp in batch],
                                   [pp.R for pp in batch], corr_path=b.CORR_IGEMM_TC)
    ctx.sync()
    for k, pair in enumerate(batch):
        g = b.results(outs[k])
        idx, sub = sample(pair, PER_PAIR, 500 + k)
        o_r, o_u, regions = cached(("mixed-bf16", k), lambda: bf16_oracle_side(orc, sub, roi=True))
        gi = {key: v[torch.from_numpy(idx).cuda()] for key, v in g.items()}
        bf16_check(gi, o_r, o_u, regions, pair.R, {})


@pytest.fixture(scope="module")
def big():
    return speckle_pair_10000()


def test_speckle_pair_10000_full_size_sampled(b, ctx, orc, big):
    pair = big
    ref16 = pair.meta["ref_u16"]
    bits = torch.from_numpy(ref16.view(np.int16)).cuda()
    pts = dev(pair.points)
    idx, sub = sample(pair, 32, 5005)
    sel = torch.from_numpy(idx).cuda()
    # F32 form
    rc = ctx.sfoc_build_u16(bits)
    sc = ctx.sfoc_build(dev(pair.sen))
    g = ctx.fastncc_match(rc, sc, pts, pair.m, pair.R, corr_path=b.CORR_DIRECT_F32)
    ctx.sync()
    o = cached(("speckle10000", 5005, 32),
               lambda: orc.match_pair(sub.ref, sub.sen, sub.points, sub.m, sub.R, want_maps=True))
    compare({k: v[sel] for k, v in g.items()}, o, pair.R, oracle_maps=o["maps"])
    assert int((g["status"] == 0).sum()) >= 0.5 * len(pair.points)
    rc.free()
    sc.free()
    # BF16 form (band tensor-core kernel: R <= 40, m + 2R = 181 > 128)
    p = b.params(dtype=b.DTYPE_BF16)
    rc = ctx.sfoc_build_u16(bits, p=p)
    sc = ctx.sfoc_build(dev(pair.sen), p=p)
    g = ctx.fastncc_match(rc, sc, pts, pair.m, pair.R, corr_path=b.CORR_IGEMM_TC)
    ctx.sync()
    o_r, o_u, regions = bf16_oracle_side(orc, sub, roi=True)
    bf16_check({k: v[sel] for k, v in g.items()}, o_r, o_u, regions, pair.R, {})
