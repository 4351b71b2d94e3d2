"""RANSAC outlier rejection (Sec. 3.2.3) on the GPU against the FP64 oracle,
through the C-ABI.  Integer results (every hypothesis's score, the winner,
the inlier set) must be identical; the final model within 1e-9 relative
(both sides solve the same systems in FP64, in different summation orders)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import apply_model, inverting_pair_512, planted_correspondences, ransac_samples  # noqa: E402


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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype else t).cuda()


def run_both(b, ctx, orc, src, dst, samp, valid=None, projective=True, tau=1.5, refits=1):
    g = ctx.fastncc_ransac(dev(src, torch.float64), dev(dst, torch.float64), dev(samp, torch.int32),
                           valid=dev(valid.astype(np.uint8)) if valid is not None else None,
                           model=b.MODEL_PROJECTIVE if projective else b.MODEL_AFFINE, threshold=tau, refits=refits,
                           want_scores=True)
    ctx.sync()
    o = orc.ransac(src, dst, samp, valid=valid, model=orc.PROJECTIVE if projective else orc.AFFINE, tau=tau,
                   refits=refits)
    return {k: v.cpu().numpy() for k, v in g.items()}, o


def check(g, o):
    np.testing.assert_array_equal(g["scores"], o["scores"])
    assert int(g["info"][0]) == o["best"]
    assert int(g["info"][1]) == o["count"]
    np.testing.assert_array_equal(g["inlier"], o["inlier"])
    scale = np.abs(o["H"]).max()
    assert np.abs(g["H"] - o["H"]).max() <= 1e-9 * scale


@pytest.mark.parametrize("projective", [True, False])
@pytest.mark.parametrize("n,frac,n_hyp,seed", [(60, 0.2, 128, 1), (1000, 0.4, 4096, 2), (4000, 0.3, 1000, 3),
                                               (257, 0.6, 333, 4)])
def test_matches_oracle_planted(b, ctx, orc, projective, n, frac, n_hyp, seed):
    src, dst, H0, out = planted_correspondences(seed, n, projective, frac, noise=0.25)
    samp = ransac_samples(seed + 50, n, n_hyp, 4 if projective else 3)
    g, o = run_both(b, ctx, orc, src, dst, samp, projective=projective)
    check(g, o)
    assert not g["inlier"][out].any()


def test_valid_mask_and_refits(b, ctx, orc):
    src, dst, H0, out = planted_correspondences(5, 500, True, 0.3, noise=0.4)
    valid = np.ones(500, bool)
    valid[::4] = False
    samp = ransac_samples(6, 500, 800, 4)
    for refits in (0, 1, 3):
        g, o = run_both(b, ctx, orc, src, dst, samp, valid=valid, refits=refits)
        check(g, o)
        assert not g["inlier"][~valid].any()


def test_degenerate_and_empty(b, ctx, orc):
    src = np.array([[0, 0], [10, 10], [20, 20], [30, 30], [5, 90.0]])
    dst = src + 3.0
    g, o = run_both(b, ctx, orc, src, dst, np.array([[0, 1, 2, 3], [1, 2, 3, 0]]))
    check(g, o)
    assert list(g["scores"]) == [-1, -1] and int(g["info"][0]) == -1
    np.testing.assert_array_equal(g["H"], np.eye(3))
    g, o = run_both(b, ctx, orc, src, dst, np.zeros((0, 4), np.int32))
    check(g, o)


def test_out_of_range_index_voids_the_hypothesis(b, ctx, orc):
    src, dst, H0, out = planted_correspondences(7, 100, True, 0.2)
    samp = ransac_samples(8, 100, 50, 4)
    bad = samp.copy()
    bad[10, 2] = 100          # one past the end
    bad[20, 0] = -1
    g = ctx.fastncc_ransac(dev(src), dev(dst), dev(bad), want_scores=True)
    sc = g["scores"].cpu().numpy()
    assert sc[10] == -1 and sc[20] == -1
    keep = np.setdiff1d(np.arange(50), [10, 20])
    o = orc.ransac(src, dst, samp[keep])
    np.testing.assert_array_equal(sc[keep], o["scores"])


def test_inverting_pair_512_matches_give_the_planted_shift(b, ctx):
    pair = inverting_pair_512()
    p = b.params(dtype=b.DTYPE_F32)
    rc = ctx.sfoc_build(dev(pair.ref), p=p)
    sc = ctx.sfoc_build(dev(pair.sen), p=p)
    pts = dev(pair.points)
    raw = ctx.fastncc_match(rc, sc, pts, pair.m, pair.R)["raw"]
    src, dst, valid = ctx.points_from_results(pts, raw)
    n = src.shape[0]
    samp = dev(ransac_samples(9, n, 2048, 4))
    g = ctx.fastncc_ransac(src, dst, samp, valid=valid)
    ctx.sync()
    H = g["H"].cpu().numpy()
    s = src.cpu().numpy()
    d = apply_model(H, s) - s                     # the model's offset at every point
    np.testing.assert_allclose(d, np.broadcast_to(pair.truth[0], d.shape), atol=0.1)
    assert int(g["info"][1]) >= 0.95 * int(valid.sum())


def test_invalid_arguments(b, ctx):
    src = dev(np.zeros((10, 2)))
    samp = dev(np.zeros((4, 4), np.int32))
    with pytest.raises(b.SfocError):
        ctx.fastncc_ransac(src, src, samp, threshold=-1.0)
    with pytest.raises(b.SfocError):
        ctx.fastncc_ransac(src, src, samp, refits=-1)
    with pytest.raises(b.SfocError):
        ctx.fastncc_ransac(src, src, samp, model=7)
