"""sfoc_build_static (the build with a fixed device scratch array and a
caller-owned output) against sfoc_build + sfoc_cube_export and against the
FP64 oracle.

Both library builds run the same steering and smoothing kernels, so the
cubes agree within the F32 cube tolerance the parity tests use (2e-5); two
calls in a row check that the scratch array left by one call does not leak
into the next.  The oracle comparison checks the static build on its own
(not only through the other GPU entry point), and the size limit is checked
at its edge.  The file name sorts last so that the test also runs after
every other GPU test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import gamma_speckle, optical_like  # noqa: E402


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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_static_build_matches_sfoc_build_twice(b, ctx):
    rng = np.random.default_rng(2024)
    images = [optical_like(rng, 300, 257), optical_like(rng, 181, 422) * gamma_speckle(rng, (181, 422), 4)]
    for img in images:
        x = dev(img)
        H, W = img.shape
        out = torch.full((12, H, W), float("nan"), dtype=torch.float32, device="cuda")
        ctx.sfoc_build_static(x, out)
        ref = ctx.sfoc_build(x).export()
        ctx.sync()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(got).all()
        np.testing.assert_allclose(got, want, rtol=0, atol=2e-5)


def test_static_build_first_order_params(b, ctx):
    rng = np.random.default_rng(5)
    img = optical_like(rng, 97, 131)
    p = b.params(n_orient=8, first_order_only=True)
    x = dev(img)
    out = torch.empty((8, 97, 131), dtype=torch.float32, device="cuda")
    ctx.sfoc_build_static(x, out, p=p)
    ref = ctx.sfoc_build(x, p=p).export()
    ctx.sync()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=2e-5)


def test_static_build_rejects_oversize_and_bf16(b, ctx):
    H, W = 2048, 2048  # 12 * 2048 * 2048 + 2 * 2048 * 2048 floats > 2^24
    x = torch.zeros((H, W), dtype=torch.float32, device="cuda")
    out = torch.empty((12, H, W), dtype=torch.float32, device="cuda")
    with pytest.raises(b.SfocError, match="static scratch"):
        ctx.sfoc_build_static(x, out)
    small = x[:64, :64].contiguous()
    out64 = torch.empty((12, 64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(b.SfocError):
        ctx.sfoc_build_static(small, out64, p=b.params(dtype=b.DTYPE_BF16))
    # an output of the wrong shape never reaches the library
    with pytest.raises(ValueError):
        ctx.sfoc_build_static(small, out)
    ctx.sync()


def test_static_build_matches_oracle(b, ctx, orc):
    """The static build against the FP64 oracle's cube (Sec. 2.1), within
    the F32 cube tolerance of the parity tests."""
    rng = np.random.default_rng(31)
    img = optical_like(rng, 90, 117)
    out = torch.empty((12, 90, 117), dtype=torch.float32, device="cuda")
    ctx.sfoc_build_static(dev(img), out)
    ctx.sync()
    want = orc.sfoc_roi(img).data
    np.testing.assert_allclose(out.cpu().numpy(), want, rtol=0, atol=2e-5)


def test_static_build_size_limit_edge(b, ctx):
    """12 channels at H = 1024: W = 1152 needs 12 * 1152 * 1024 + 2 * 1024 *
    1152 = 16,515,072 floats of the 2^24 and is built (same cube as
    sfoc_build); W = 1153 pads its planes to 1184 floats a row, needs
    16,910,336 and is refused before any kernel runs."""
    rng = np.random.default_rng(8)
    H = 1024
    img = optical_like(rng, H, 1153)
    x = dev(img[:, :1152])
    out = torch.empty((12, H, 1152), dtype=torch.float32, device="cuda")
    ctx.sfoc_build_static(x, out)
    ref = ctx.sfoc_build(x).export()
    ctx.sync()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=0, atol=2e-5)
    x2 = dev(img)
    out2 = torch.empty((12, H, 1153), dtype=torch.float32, device="cuda")
    with pytest.raises(b.SfocError) as e:
        ctx.sfoc_build_static(x2, out2)
    assert e.value.code == -6 and "16910336" in str(e.value)
    ctx.sync()
