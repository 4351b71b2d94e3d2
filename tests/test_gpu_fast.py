"""Block-based FAST (Sec. 3.1.1) on the GPU against the oracle, through the
C-ABI.  Scores are FP32 differences of the stored pixels on both sides, so
points and scores must be identical."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import sar_pair_2048, optical_like  # noqa: E402


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


def gpu_fast(ctx, img, t, gy, gx, margin):
    pts, sc = ctx.fast_blocks(torch.from_numpy(np.ascontiguousarray(img, np.float32)).cuda(), t, gy, gx, margin)
    ctx.sync()
    return pts.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("H,W,gy,gx,t,margin,seed", [
    (77, 93, 3, 4, 0.05, 3, 1),        # ragged, uneven partition
    (130, 33, 7, 2, 0.02, 5, 2),
    (512, 512, 8, 8, 0.05, 20, 3),
    (300, 700, 2, 3, 0.08, 3, 4),      # blocks of 150 x 233: several sub-tiles each
    (64, 64, 64, 64, 0.0, 0, 5),       # one pixel per block, threshold 0
])
def test_matches_oracle(b, ctx, orc, H, W, gy, gx, t, margin, seed):
    rng = np.random.default_rng(seed)
    img = optical_like(rng, H, W) if seed % 2 else rng.random((H, W)).astype(np.float32)
    g = gpu_fast(ctx, img, t, gy, gx, margin)
    o = orc.fast_blocks(img, t, gy, gx, margin)
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])


def test_full_size_reference(b, ctx, orc):
    """The 2048^2 reference of the benchmark workload, 32 x 32 blocks."""
    img = sar_pair_2048().ref
    g = gpu_fast(ctx, img, 0.05, 32, 32, 61)
    o = orc.fast_blocks(img, 0.05, 32, 32, 61)
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])
    assert (g[0][:, 0] >= 0).mean() > 0.8   # the margin empties most of the outer ring of blocks


def test_flat_and_margin(b, ctx, orc):
    img = np.full((100, 120), 0.4, np.float32)
    p, s = gpu_fast(ctx, img, 0.05, 4, 4, 3)
    assert (p == -1).all() and (s == 0).all()
    img = optical_like(np.random.default_rng(9), 100, 120)
    p, s = gpu_fast(ctx, img, 0.05, 2, 2, 60)     # the margin leaves no candidates
    assert (p == -1).all()


def test_invalid_arguments(b, ctx):
    img = torch.zeros((50, 60), dtype=torch.float32, device="cuda")
    for kw in (dict(grid_y=0), dict(grid_x=61), dict(margin=-1), dict(threshold=-0.1), dict(threshold=float("inf"))):
        with pytest.raises(b.SfocError):
            ctx.fast_blocks(img, **{"threshold": 0.05, "grid_y": 2, "grid_x": 2, "margin": 3, **kw})
