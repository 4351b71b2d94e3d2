"""GPU path against the FP64 oracle, element by element, through the C ABI.

Sizes span several kernel tiles plus ragged tails; the full-size workload
(2048^2, 1000 points, m=81, R=20) runs in the same launch configuration as
the benchmark and is checked on a seeded sample of points the oracle
computes one by one.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import inverting_pair_512, sar_pair_2048, tiny_pair  # noqa: E402

from parity import cached, compare  # noqa: E402


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
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ---------------------------------------------------------------------------
# SFOC cube (Sec. 2.1)
# ---------------------------------------------------------------------------

CUBE_ATOL = 2e-5   # FP32 filtering of [0,1] images, values normalised to <= 1


@pytest.mark.parametrize("H,W,seed", [(77, 93, 1), (33, 130, 2), (512, 512, 3)])
def test_cube_f32_matches_oracle(b, ctx, orc, H, W, seed):
    rng = np.random.default_rng(seed)
    from workloads import optical_like
    img = optical_like(rng, H, W)
    cube = ctx.sfoc_build(dev(img))
    got = cube.export().cpu().numpy().astype(np.float64)
    want = orc.sfoc_roi(img).data
    err = np.abs(got - want)
    assert err.max() <= CUBE_ATOL, "max err %g at %s" % (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_cube_variants_match_oracle(b, ctx, orc):
    rng = np.random.default_rng(4)
    img = rng.random((45, 70)).astype(np.float32)
    for kw in (dict(first_order_only=True), dict(rectify=False), dict(scales=(1.0, 2.0, 3.0)),
               dict(n_orient=4, dil=(1, 2)), dict(eps=0.05)):
        okw = dict(kw)
        p = b.params(**kw)
        got = ctx.sfoc_build(dev(img), p=p).export().cpu().numpy()
        want = orc.sfoc_roi(img, orc.params(**okw)).data
        assert np.abs(got - want).max() <= CUBE_ATOL, kw


def _group_norm_tol(orc, img, kw):
    """Per-value bound for a cube whose groups may be unsmoothed: the FP32
    error of a pre-normalisation value (at most 1e-6 here) is divided by
    ||D|| + eps in the group normalisation, so a group with a small norm
    gets 1e-6 / (||D|| + eps) on top of CUBE_ATOL.  D is the oracle's
    pre-normalisation input (eps = 1e30 makes the normalisation an exact
    division by 1e30)."""
    p = orc.params(eps=1e30, **kw)
    D = orc.sfoc_roi(img, p).data * 1e30
    no = 6
    nrm = np.concatenate([np.repeat(np.linalg.norm(D[g * no:(g + 1) * no], axis=0)[None], no, 0)
                          for g in range(D.shape[0] // no)])
    return CUBE_ATOL + 1e-6 / (nrm + 1e-3)


SMOOTHING_VARIANTS = [dict(sigma_d1=0.0, sigma_d2=0.0), dict(sigma_d1=0.0), dict(dil=(1,)),
                      dict(dil=(2,), sigma_d2=0.0)]


@pytest.mark.parametrize("kw", SMOOTHING_VARIANTS, ids=["unsmoothed", "first_unsmoothed", "plain_gauss",
                                                        "rate2_second_unsmoothed"])
def test_cube_smoothing_variants_match_oracle(b, ctx, orc, kw):
    """The smoothing variants of Fig. 3 (Sec. 2.1): unsmoothed groups
    (sigma_d = 0), a plain Gaussian (one rate, r = 1), a single other rate."""
    rng = np.random.default_rng(4)
    img = rng.random((45, 70)).astype(np.float32)
    got = ctx.sfoc_build(dev(img), p=b.params(**kw)).export().cpu().numpy().astype(np.float64)
    want = orc.sfoc_roi(img, orc.params(**kw)).data
    tol = _group_norm_tol(orc, img, kw)
    err = np.abs(got - want)
    assert np.all(err <= tol), "max err %g (tol there %g)" % (err.max(), tol.flat[err.argmax()])


def test_negative_smoothing_std_is_rejected(b, ctx):
    img = np.zeros((40, 40), np.float32)
    with pytest.raises(b.SfocError):
        ctx.sfoc_build(dev(img), p=b.params(sigma_d2=-1.0))

def test_integral_planes(b, ctx, orc):
    """Eq. 14: exclusive prefix of the channel sums.  The library keeps exact
    64-bit sums of each pixel's value rounded to a multiple of 2^-28, so an
    entry covering n pixels is within n * 2^-29 of the FP64 prefix (plus the
    FP32 rounding of the sum planes themselves, relative 2^-23 per pixel), and
    an entry whose rectangle holds a NaN cube value is NaN."""
    rng = np.random.default_rng(5)
    from workloads import optical_like
    for H, W, nan_at in ((77, 93, None), (200, 131, (120, 60))):
        img = optical_like(rng, H, W)
        if nan_at is not None:
            img[nan_at] = np.nan
        cube = ctx.sfoc_build(dev(img))
        P = cube.export_integral().cpu().numpy()
        c = cube.export().cpu().numpy().astype(np.float64)
        npx = np.arange(H + 1)[:, None] * np.arange(W + 1)[None, :]
        for k, plane in enumerate((c.sum(0), (c * c).sum(0))):
            want = orc.integral(plane)
            assert np.array_equal(np.isnan(P[k]), np.isnan(want))
            ok = ~np.isnan(want)
            absw = orc.integral(np.abs(np.nan_to_num(plane)))
            bound = npx * 2.0 ** -29 + 2.0 ** -22 * absw + 1e-12
            assert np.all(np.abs(P[k] - want)[ok] <= bound[ok])


# ---------------------------------------------------------------------------
# matching (Sec. 2.2, Eq. 8-16)
# ---------------------------------------------------------------------------

F32_PATHS = ["direct", "fft"]


def f32_path(b, name):
    return {"direct": b.CORR_DIRECT_F32, "fft": b.CORR_FFT}[name]


def gpu_match(ctx, b, pair, p=None, corr=0, want_maps=False):
    rc = ctx.sfoc_build(dev(pair.ref), p=p)
    sc = ctx.sfoc_build(dev(pair.sen), p=p)
    return ctx.fastncc_match(rc, sc, dev(pair.points), pair.m, pair.R, corr_path=corr, want_maps=want_maps)


@pytest.mark.parametrize("path", F32_PATHS)
def test_match_inverting_pair_512_f32(b, ctx, orc, path):
    pair = inverting_pair_512()
    o = orc.match_pair(pair.ref, pair.sen, pair.points, pair.m, pair.R, want_maps=True, roi=False)
    g = gpu_match(ctx, b, pair, corr=f32_path(b, path), want_maps=True)
    st = compare(g, o, pair.R, oracle_maps=o["maps"])
    # the NCC maps themselves agree everywhere
    gm = g["maps"].cpu().numpy()
    assert np.abs(gm - o["maps"]).max() <= 1e-4
    assert st["valid"] == 100


@pytest.mark.parametrize("H,W,m,R,npts,seed", [
    (70, 83, 9, 4, 12, 11),     # ragged, small
    (96, 61, 10, 3, 9, 12),     # even template
    (64, 64, 1, 2, 16, 13),     # m = 1
    (60, 75, 15, 0, 9, 14),     # R = 0
    (150, 140, 31, 12, 20, 15),
    (120, 130, 24, 20, 10, 16),  # m + 2R = 64: the smallest transform's edge
    (200, 210, 65, 31, 6, 17),   # m + 2R = 127
])
@pytest.mark.parametrize("path", F32_PATHS)
def test_match_small_cases(b, ctx, orc, H, W, m, R, npts, seed, path):
    pair = tiny_pair(seed, H, W, m, R, npts, shift=(2, -1))
    o = orc.match_pair(pair.ref, pair.sen, pair.points, m, R, want_maps=True, roi=False)
    g = gpu_match(ctx, b, pair, corr=f32_path(b, path), want_maps=True)
    compare(g, o, R, oracle_maps=o["maps"])


@pytest.mark.parametrize("kw", [dict(first_order_only=True), dict(sigma_d1=0.0, sigma_d2=0.0), dict(dil=(1,))],
                         ids=["f_sfoc", "unsmoothed", "plain_gauss"])
@pytest.mark.parametrize("path", F32_PATHS)
def test_match_descriptor_variants(b, ctx, orc, kw, path):
    """Matching on the variant cubes (F-SFOC's 6 channels, Sec. 4.2; the
    smoothings of Fig. 3).  An unsmoothed cube's larger error at small-norm
    pixels (up to about 1e-4) moves NCC by |dS| / |S - mean S| ~ 1e-5 over
    a 21 x 21 x z window, inside the 1e-4 target."""
    pair = tiny_pair(31, 120, 130, 21, 8, 12, shift=(3, -2))
    o = orc.match_pair(pair.ref, pair.sen, pair.points, pair.m, pair.R, p=orc.params(**kw), want_maps=True,
                       roi=False)
    g = gpu_match(ctx, b, pair, p=b.params(**kw), corr=f32_path(b, path), want_maps=True)
    st = compare(g, o, pair.R, oracle_maps=o["maps"])
    assert st["valid"] >= 8

@pytest.mark.parametrize("path", F32_PATHS)
def test_status_cases(b, ctx, orc, path):
    """Out-of-bounds points, a flat template and a NaN pixel."""
    pair = tiny_pair(21, 90, 90, 11, 5, 4)
    sen = pair.sen.copy()
    sen[0:60, 40:90] = 0.5             # flat up to the border -> zero cube -> FLAT_TEMPLATE
    sen[70, 20] = np.nan               # NaN propagates to nearby cube values
    # points are (x, y)
    pts = np.array([[3, 45], [45, 87], [65, 28], [20, 70], [30, 45], [22, 68]], np.int32)
    pair.sen = sen
    pair.points = pts
    o = orc.match_pair(pair.ref, sen, pts, 11, 5, want_maps=True, roi=False)
    assert set(o["status"].tolist()) >= {1, 2, 4}
    g = gpu_match(ctx, b, pair, corr=f32_path(b, path), want_maps=True)
    compare(g, o, 5, oracle_maps=o["maps"])


@pytest.mark.parametrize("path", F32_PATHS)
def test_sar_pair_2048_full_size_sampled(b, ctx, orc, path):
    """2048^2, 1000 points, m=81, R=20: the benchmark's configuration; the
    oracle checks a seeded sample of 64 points (about 12 s of oracle work,
    shared by both paths)."""
    pair = cached("sar2048", sar_pair_2048)
    g = gpu_match(ctx, b, pair, corr=f32_path(b, path))
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(len(pair.points), 64, replace=False))
    o = cached(("sar2048-oracle", 2024, 64),
               lambda: orc.match_pair(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R, want_maps=True))
    gs = {k: v[torch.from_numpy(idx).cuda()] for k, v in g.items()}
    compare(gs, o, pair.R, oracle_maps=o["maps"])
    assert int((g["status"] == 0).sum()) >= 900


def test_host_entry_matches_device(b, ctx):
    pair = inverting_pair_512()
    p = b.params()
    raw_d = ctx.register_pair(dev(pair.ref), dev(pair.sen), dev(pair.points), pair.m, pair.R, p=p)
    raw_h = ctx.register_pair_host(torch.from_numpy(pair.ref).pin_memory(), torch.from_numpy(pair.sen).pin_memory(),
                                   torch.from_numpy(pair.points).pin_memory(), pair.m, pair.R, p=p)
    assert torch.equal(raw_d.cpu(), raw_h)


def test_invalid_arguments_return_errors(b, ctx):
    pair = tiny_pair(31, 60, 60, 9, 3, 4)
    rc = ctx.sfoc_build(dev(pair.ref))
    sc = ctx.sfoc_build(dev(pair.sen))
    with pytest.raises(b.SfocError) as e:
        ctx.fastncc_match(rc, sc, dev(pair.points), 0, 3)
    assert e.value.code == -1
    with pytest.raises(b.SfocError) as e:
        ctx.fastncc_match(rc, sc, dev(pair.points), 9, 3, corr_path=b.CORR_IGEMM_TC)
    assert e.value.code == -6
    with pytest.raises(b.SfocError):
        ctx.sfoc_build(dev(pair.ref), p=b.params(n_orient=9))


def test_empty_point_sets(b, ctx):
    """n = 0 through every matching entry point and path: nothing to match,
    status OK, no result rows (empty inputs)."""
    pair = tiny_pair(41, 60, 70, 9, 3, 4)
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    rc, sc = ctx.sfoc_build(dev(pair.ref)), ctx.sfoc_build(dev(pair.sen))
    for corr in (b.CORR_AUTO, b.CORR_FFT, b.CORR_DIRECT_F32):
        assert ctx.fastncc_match(rc, sc, empty, 9, 3, corr_path=corr)["raw"].shape == (0, 6)
    p16 = b.params(dtype=b.DTYPE_BF16)
    rb, sb = ctx.sfoc_build(dev(pair.ref), p=p16), ctx.sfoc_build(dev(pair.sen), p=p16)
    assert ctx.fastncc_match(rb, sb, empty, 9, 3, corr_path=b.CORR_IGEMM_TC)["raw"].shape == (0, 6)
    assert ctx.register_pair(dev(pair.ref), dev(pair.sen), empty, 9, 3).shape == (0, 6)
    outs = ctx.fastncc_match_batch([rc, rc], [sc, sc], [empty, dev(pair.points)], [9, 9], [3, 3])
    ctx.sync()
    assert outs[0].shape == (0, 6) and outs[1].shape == (len(pair.points), 6)


@pytest.mark.parametrize("m,R,path", [
    (129, 2, "auto"),       # m beyond the API's 128
    (9, 64, "auto"),        # R beyond the API's 63
    (128, 63, "direct"),    # the direct kernel's staged window (254 x 256 floats) exceeds shared memory
    (9, 60, "fft"),         # m + 2R = 129 > 128: no transform size
])
def test_sizes_past_the_limits_are_refused(b, ctx, m, R, path):
    """Sizes past the API's or a form's limits return SFOC_ERR_UNSUPPORTED
    before any correlation kernel runs, and the context stays usable."""
    pair = tiny_pair(43, 80, 80, 9, 3, 4)
    rc, sc = ctx.sfoc_build(dev(pair.ref)), ctx.sfoc_build(dev(pair.sen))
    corr = {"auto": b.CORR_AUTO, "direct": b.CORR_DIRECT_F32, "fft": b.CORR_FFT}[path]
    with pytest.raises(b.SfocError) as e:
        ctx.fastncc_match(rc, sc, dev(pair.points), m, R, corr_path=corr)
    assert e.value.code == -6
    ctx.sync()
    assert ctx.fastncc_match(rc, sc, dev(pair.points), 9, 3)["raw"].shape == (len(pair.points), 6)

def test_allocation_failure_is_reported_and_the_context_recovers(b, ctx):
    """A workspace no device can hold: sfoc_ctx_reserve returns SFOC_ERR_OOM,
    the failed allocation leaves no error behind, and the next match on the
    same context regrows its workspace and succeeds."""
    pair = tiny_pair(45, 70, 70, 9, 3, 6)
    rc, sc = ctx.sfoc_build(dev(pair.ref)), ctx.sfoc_build(dev(pair.sen))
    with pytest.raises(b.SfocError) as e:
        ctx.reserve(1 << 50)
    assert e.value.code == -3
    g = ctx.fastncc_match(rc, sc, dev(pair.points), pair.m, pair.R)
    ctx.sync()
    assert int((g["status"] == 0).sum()) > 0

def test_binding_checks_shapes_before_the_library(b, ctx):
    """Tensors whose shape does not match the sizes the binding passes are
    refused in Python, before the library could read past their end."""
    pair = tiny_pair(46, 60, 60, 9, 3, 4)
    rc, sc = ctx.sfoc_build(dev(pair.ref)), ctx.sfoc_build(dev(pair.sen))
    flat = dev(pair.points).reshape(-1).contiguous()
    with pytest.raises(ValueError):
        ctx.fastncc_match(rc, sc, flat, 9, 3)
    with pytest.raises(ValueError):
        ctx.register_pair(dev(pair.ref), dev(pair.sen), dev(pair.points), 9, 3,
                          out=torch.empty((1, 6), dtype=torch.int32, device="cuda"))
    src = torch.zeros((10, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        ctx.fastncc_ransac(src, src, torch.zeros((4, 3), dtype=torch.int32, device="cuda"))   # projective: 4 wide
    with pytest.raises(ValueError):
        ctx.rectify(dev(pair.ref), torch.eye(3, dtype=torch.float64, device="cuda").reshape(-1))
    ctx.sync()

def test_u16_input_matches_scaled_float(b, ctx, orc):
    """sfoc_build_u16: a 16-bit image is read as v / 65535 (the input step
    of the 10000^2 workload); the cube equals the oracle's on the FP64
    scaled image and the GPU cube of the float32 image v / 65535."""
    rng = np.random.default_rng(21)
    from workloads import optical_like
    img16 = np.round(optical_like(rng, 83, 97) * 65535.0).astype(np.uint16)
    bits = torch.from_numpy(img16.view(np.int16)).cuda()
    cube16 = ctx.sfoc_build_u16(bits)
    f = (img16.astype(np.float32) / np.float32(65535.0)).astype(np.float32)
    cubef = ctx.sfoc_build(torch.from_numpy(f).cuda())
    got16 = cube16.export().cpu().numpy()
    gotf = cubef.export().cpu().numpy()
    np.testing.assert_array_equal(got16, gotf)
    want = orc.sfoc_roi(img16.astype(np.float64) / 65535.0).data
    np.testing.assert_allclose(got16, want, rtol=0, atol=2e-5)


def test_cube_view_layouts(b, ctx):
    rng = np.random.default_rng(22)
    from workloads import optical_like
    img = torch.from_numpy(optical_like(rng, 40, 52)).cuda()
    for dt in (b.DTYPE_F32, b.DTYPE_BF16):
        cube = ctx.sfoc_build(img, p=b.params(dtype=dt))
        addr, z, H, W, pitch, dtype = cube.view()
        assert (z, H, W, dtype) == (12, 40, 52, dt) and addr
        exp = cube.export()
        ctx.sync()

        class _View:  # zero-copy tensor over the viewed device memory
            def __init__(self, shape, typestr):
                self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (addr, False),
                                                 "version": 3}

        if dt == b.DTYPE_F32:
            raw = torch.as_tensor(_View((z, H, pitch), "<f4"), device="cuda")
            assert torch.equal(raw[:, :, :W], exp)
        else:
            raw = torch.as_tensor(_View((2, H, W, 8), "<i2"), device="cuda").view(torch.bfloat16)
            chans = torch.cat([raw[0, :, :, :6], raw[1, :, :, :6]], dim=-1).permute(2, 0, 1).float()
            assert torch.equal(chans, exp)
            assert torch.all(raw[:, :, :, 6:] == 0)


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(b, ctx):
    """The failure path of the tensor-core kernels on a GPU: a bounded wait
    (1 ms) on a barrier nothing arrives on expires, the kernel frees its
    tensor memory, sets the context's error word and returns; sync reports
    SFOC_ERR_TIMEOUT once, the word is cleared, and a BF16 tensor-core match
    on the same context then runs normally."""
    ctx.sync()
    ctx.selftest_timeout(1000)
    with pytest.raises(b.SfocError) as e:
        ctx.sync()
    assert e.value.code == -5
    ctx.sync()  # the error word was cleared
    pair = tiny_pair(45, 90, 96, 15, 4, 6, shift=(1, 1))
    p = b.params(dtype=b.DTYPE_BF16)
    rc, sc = ctx.sfoc_build(dev(pair.ref), p=p), ctx.sfoc_build(dev(pair.sen), p=p)
    res = ctx.fastncc_match(rc, sc, dev(pair.points), pair.m, pair.R, corr_path=b.CORR_TC_BAND)
    ctx.sync()
    assert int((res["status"] == 0).sum()) + int((res["status"] == 3).sum()) > 0
    with pytest.raises(b.SfocError):
        ctx.selftest_timeout(0)  # a limit out of range is refused before any launch
