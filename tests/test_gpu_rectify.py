"""Rectification (Sec. 3.2.3) on the GPU against the oracle: the same model
in, fill positions identical, values within a few float ulps (the GPU maps
in FP64 and blends in FP32, the oracle blends in double)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import optical_like, planted_model  # noqa: E402


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


def run(ctx, img, H, out_shape=None, fill=-1.0):
    g = ctx.rectify(torch.from_numpy(img).cuda(), torch.from_numpy(np.asarray(H, np.float64)).cuda(),
                    out_shape=out_shape, fill=fill)
    ctx.sync()
    return g.cpu().numpy()


@pytest.mark.parametrize("kind,shape,out_shape,seed", [
    ("identity", (37, 53), None, 1),
    ("shift", (90, 70), (100, 80), 2),
    ("affine", (256, 300), None, 3),
    ("projective", (511, 389), (400, 450), 4),
])
def test_matches_oracle(b, ctx, orc, kind, shape, out_shape, seed):
    rng = np.random.default_rng(seed)
    img = optical_like(rng, *shape)
    if kind == "identity":
        H = np.eye(3)
    elif kind == "shift":
        H = np.array([[1, 0, 7], [0, 1, -4], [0, 0, 1.0]])
    else:
        H = planted_model(rng, projective=kind == "projective")
    g = run(ctx, img, H, out_shape)
    o = orc.rectify(img, H, out_shape=out_shape, fill=-1.0)
    np.testing.assert_array_equal(g == -1.0, o == -1.0)
    assert np.abs(g - o).max() <= 5e-7


def test_singular_model_fills(b, ctx):
    img = np.ones((20, 30), np.float32)
    g = run(ctx, img, np.zeros((3, 3)), fill=0.25)
    assert (g == 0.25).all()


def test_invalid_arguments(b, ctx):
    img = torch.zeros((10, 10), dtype=torch.float32, device="cuda")
    m = torch.eye(3, dtype=torch.float64, device="cuda")
    with pytest.raises(b.SfocError):
        ctx.rectify(img, m, out_shape=(0, 10))
