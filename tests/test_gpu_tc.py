"""BF16 form: the tcgen05 correlation kernel against the FP64 oracle.

Kernel parity: the oracle's FP64 cube rounded to bf16 (round to nearest
even, a plain definition) is matched by the oracle's Eq. 8; the GPU's BF16
form must agree with it.  The GPU rounds its FP32 cube, which is within
2e-5 of the oracle's, so values that close to a rounding midpoint may round
the other way (one ulp).  Tolerances: per point at the best offset,
1e-4 + 6 sigma of the NCC change those flips imply through the exact NCC
gradient (parity.flip_tolerance); over whole maps, the worst case
1e-4 + ||delta_S||/sigma_S + ||delta_T||/sigma_T (parity.ncc_rounding_bound).
Offsets must agree wherever the oracle's top-2 margin exceeds twice the
point tolerance.

Precision report: the same GPU results against the oracle on the unrounded
FP64 cube; the error must stay inside the storage bound
1e-4 + 2^-9 (||S||/sigma_S + ||T||/sigma_T) (parity.storage_bound).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from workloads import inverting_pair_512, sar_pair_2048, tiny_pair  # noqa: E402

from parity import bf16_check as check, bf16_oracle_side as oracle_side, cached  # noqa: E402


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


def gpu_bf16(ctx, b, pair, want_maps=False, path=None):
    p = b.params(dtype=b.DTYPE_BF16)
    rc = ctx.sfoc_build(dev(pair.ref), p=p)
    sc = ctx.sfoc_build(dev(pair.sen), p=p)
    return ctx.fastncc_match(rc, sc, dev(pair.points), pair.m, pair.R,
                             corr_path=b.CORR_IGEMM_TC if path is None else path, want_maps=want_maps)


# "auto": IGEMM_TC, the measured fastest tensor-core form; "fft": the Fourier
# correlation reading the bf16 cube; "any": AUTO, the fastest of all of them
FORMS = ["auto", "toeplitz", "column", "band", "fft", "any"]


def form_path(b, form):
    return {"auto": None, "toeplitz": b.CORR_TC_TOEPLITZ, "column": b.CORR_TC_COLUMN,
            "band": b.CORR_TC_BAND, "fft": b.CORR_FFT, "any": b.CORR_AUTO}[form]


SMALL = [
    (70, 83, 9, 4, 12, 11),
    (96, 61, 10, 3, 9, 12),     # even template
    (64, 64, 1, 2, 16, 13),     # m = 1
    (60, 75, 15, 0, 9, 14),     # R = 0
    (150, 140, 31, 12, 20, 15),
    (110, 120, 17, 7, 25, 16),
    (190, 200, 64, 31, 8, 17),  # m + 2R = 126: column form, 4 offsets per group
]


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("H,W,m,R,npts,seed", SMALL)
def test_tc_small_cases(b, ctx, orc, H, W, m, R, npts, seed, form):
    """Every correlation form of BF16 cubes on the same inputs: the column
    form (m + 2R <= 128), the Toeplitz form, the band form and the Fourier
    correlation of the bf16 values, and the two measured choices."""
    pair = tiny_pair(seed, H, W, m, R, npts, shift=(2, -1))
    g = gpu_bf16(ctx, b, pair, want_maps=True, path=form_path(b, form))
    ctx.sync()
    o_r, o_u, regions = oracle_side(orc, pair)
    check(g, o_r, o_u, regions, R, {})


@pytest.mark.parametrize("form", ["auto", "band"])
@pytest.mark.parametrize("H,W,m,R,npts,seed", [
    (230, 240, 61, 35, 8, 18),   # m + 2R = 131: no column form
    (200, 190, 101, 14, 6, 19),  # m + 2R = 129
    (260, 250, 101, 40, 4, 20),  # the largest radius of the band form
])
def test_tc_wide_windows(b, ctx, orc, H, W, m, R, npts, seed, form):
    pair = tiny_pair(seed, H, W, m, R, npts, shift=(-3, 2))
    g = gpu_bf16(ctx, b, pair, want_maps=True, path=form_path(b, form))
    ctx.sync()
    o_r, o_u, regions = oracle_side(orc, pair)
    check(g, o_r, o_u, regions, R, {})


@pytest.mark.parametrize("kw", [dict(), dict(sigma_d1=0.0, sigma_d2=0.0), dict(dil=(1,))],
                         ids=["paper", "unsmoothed", "plain_gauss"])
def test_bf16_cube_is_rounded_oracle_cube(b, ctx, orc, kw):
    rng = np.random.default_rng(3)
    from workloads import optical_like
    img = optical_like(rng, 77, 93)
    cube = ctx.sfoc_build(dev(img), p=b.params(dtype=b.DTYPE_BF16, **kw))
    got = cube.export().cpu().numpy().astype(np.float64)
    want = orc.sfoc_roi(img, orc.params(**kw)).data
    # one bf16 rounding (half an ulp: 2^-9 relative) on top of the FP32
    # error, which an unsmoothed group's small norm amplifies (see
    # test_gpu_parity._group_norm_tol: 1e-6 / (||D|| + eps))
    D = orc.sfoc_roi(img, orc.params(eps=1e30, **kw)).data * 1e30
    nrm = np.concatenate([np.repeat(np.linalg.norm(D[g * 6:(g + 1) * 6], axis=0)[None], 6, 0) for g in (0, 1)])
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 2e-5 + 1e-6 / (nrm + 1e-3))


@pytest.mark.parametrize("form", FORMS)
def test_tc_inverting_pair_512(b, ctx, orc, form):
    pair = inverting_pair_512()
    g = gpu_bf16(ctx, b, pair, want_maps=True, path=form_path(b, form))
    ctx.sync()
    o_r, o_u, regions = oracle_side(orc, pair)
    rep = {}
    st = check(g, o_r, o_u, regions, pair.R, rep)
    assert st["valid"] == 100
    assert rep["bf16_vs_fp64_offsets_equal"] >= 95


@pytest.mark.parametrize("form", ["auto", "band", "fft"])
def test_tc_sar_pair_2048_full_size_sampled(b, ctx, orc, form):
    """2048^2, 1000 points, m=81, R=20 in the benchmark's launch
    configuration; a seeded sample of 64 points against the oracle (shared by
    both forms)."""
    pair = cached("sar2048", sar_pair_2048)
    g = gpu_bf16(ctx, b, pair, path=form_path(b, form))
    ctx.sync()
    rng = np.random.default_rng(77)
    idx = np.sort(rng.choice(len(pair.points), 64, replace=False))
    sub = type(pair)(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R, pair.truth[idx])
    o_r, o_u, regions = cached(("sar2048-bf16-oracle", 77, 64), lambda: oracle_side(orc, sub, roi=True))
    gs = {k: v[torch.from_numpy(idx).cuda()] for k, v in g.items()}
    check(gs, o_r, o_u, regions, pair.R, {})
    assert int((g["status"] == 0).sum()) >= 900


@pytest.mark.parametrize("m,R,path", [
    (20, 60, "column"),     # m + 2R = 140 > 128: no column form
    (61, 41, "band"),       # R = 41: N = 112 rows, past the band form's 96
])
def test_forced_forms_past_their_limits_are_refused(b, ctx, m, R, path):
    """Forcing a tensor-core form outside its limits returns
    SFOC_ERR_UNSUPPORTED before the kernel runs; the context stays usable."""
    pair = tiny_pair(44, 90, 90, 9, 3, 4)
    p = b.params(dtype=b.DTYPE_BF16)
    rc, sc = ctx.sfoc_build(dev(pair.ref), p=p), ctx.sfoc_build(dev(pair.sen), p=p)
    with pytest.raises(b.SfocError) as e:
        ctx.fastncc_match(rc, sc, dev(pair.points), m, R, corr_path=form_path(b, path))
    assert e.value.code == -6
    ctx.sync()
    assert ctx.fastncc_match(rc, sc, dev(pair.points), 9, 3)["raw"].shape == (len(pair.points), 6)
