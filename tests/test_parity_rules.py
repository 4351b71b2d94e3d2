"""The comparison rules of the GPU parity tests, checked on the CPU.

The BF16 form is judged with tolerances derived in tests/parity.py from the
rounding it performs.  These tests pin each rule to something outside it:
the rounding helper against torch's own bfloat16 conversion, the ulp helper
against the spacing of representable values, and every NCC bound against
brute-force Pearson correlations of perturbed windows (Eq. 8 is the Pearson
correlation of the flattened windows).
"""
import numpy as np
import pytest

from parity import (bf16_round, bf16_ulp, compare, flip_tolerance, ncc_rounding_bound, storage_bound,
                    subpixel_tol)

torch = pytest.importorskip("torch")


def _torch_bf16(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_round_is_torch_conversion():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 4, 20000),
                        rng.random(5000)]).astype(np.float32)
    np.testing.assert_array_equal(bf16_round(x), _torch_bf16(x))
    # exact ties (low 16 bits 0x8000) go to the even neighbour, both signs
    base = (rng.integers(0x3000, 0x4800, 4000).astype(np.uint32) << 16) | 0x8000
    ties = base.view(np.float32)
    ties = np.concatenate([ties, -ties])
    np.testing.assert_array_equal(bf16_round(ties), _torch_bf16(ties))
    assert np.all((bf16_round(ties).astype(np.float32).view(np.uint32) >> 16) % 2 == 0)


def test_bf16_ulp_is_the_spacing():
    rng = np.random.default_rng(1)
    v = bf16_round(rng.random(3000) * 10.0 ** rng.integers(-4, 3, 3000))
    u = bf16_ulp(v)
    # the next value up is representable, nothing lies strictly between
    np.testing.assert_array_equal(bf16_round(v + u), v + u)
    np.testing.assert_array_equal(bf16_round(v + 0.49 * u), v)
    # 8 significant bits: u / v in (2^-8, 2^-7]
    r = u / v
    assert np.all((r > 2.0 ** -8) & (r <= 2.0 ** -7))


def _pearson_maps(S, T):
    """NCC (Eq. 8) of T against every m x m window of S, by brute force."""
    z, m = T.shape[0], T.shape[1]
    P = S.shape[1] - m + 1
    t = (T - T.mean()).ravel()
    out = np.empty((P, P))
    for dy in range(P):
        for dx in range(P):
            s = S[:, dy:dy + m, dx:dx + m].ravel()
            s = s - s.mean()
            out[dy, dx] = s @ t / (np.linalg.norm(s) * np.linalg.norm(t))
    return out


def _cube(rng, z, n):
    # values like a normalised cube: non-negative, below 1
    return rng.random((z, n, n)) * rng.random((z, 1, 1))


@pytest.mark.parametrize("lo,hi,err", [(0.25, 1.0, 5e-4),   # every ulp above 2 cube_err: one-ulp flips
                                        (1e-4, 4e-3, 2e-5),   # ulps near or below cube_err: several
                                        (0.0, 1.0, 2e-5)],    # the cube's range at the tests' cube_err
                         ids=["large", "tiny", "cube"])
@pytest.mark.parametrize("seed", [2, 3, 4])
def test_rounding_bound_covers_cube_differences(seed, lo, hi, err):
    """Two cubes within cube_err of each other (the GPU's FP32 cube and the
    oracle's FP64 one), each rounded to bf16, give NCC maps (Eq. 8) within
    ncc_rounding_bound at every offset (its base is the FP32 allowance, not
    needed here)."""
    rng = np.random.default_rng(seed)
    z, m, R = 3, 6, 3
    S = rng.uniform(lo, hi, (z, m + 2 * R, m + 2 * R))
    T = rng.uniform(lo, hi, (z, m, m))
    S2 = S + rng.uniform(-err, err, S.shape)
    T2 = T + rng.uniform(-err, err, T.shape)
    a = _pearson_maps(bf16_round(S), bf16_round(T))
    b = _pearson_maps(bf16_round(S2), bf16_round(T2))
    bound = ncc_rounding_bound(S, T, cube_err=err, base=0.0)
    assert np.all(np.abs(b - a) <= bound)
    assert np.abs(b - a).max() > 0          # the case is not vacuous


@pytest.mark.parametrize("seed", [5, 6])
def test_storage_bound_covers_bf16_storage(seed):
    """Eq. 8 on the bf16-rounded cubes stays within storage_bound of Eq. 8
    on the exact cubes at every offset."""
    rng = np.random.default_rng(seed)
    z, m, R = 4, 7, 2
    S = _cube(rng, z, m + 2 * R)
    T = _cube(rng, z, m)
    exact = _pearson_maps(S, T)
    rounded = _pearson_maps(bf16_round(S), bf16_round(T))
    bound = storage_bound(S, T, base=0.0)
    assert np.all(np.abs(rounded - exact) <= bound)
    # and it is not vacuous: the bound is below 5 % of the NCC range here
    assert bound.max() < 0.1


def test_flip_tolerance_covers_single_flips():
    """Moving one ambiguous value by one ulp changes NCC by about |g_i| ulp_i,
    which the 6-sigma flip tolerance covers."""
    rng = np.random.default_rng(7)
    z, m, err = 3, 8, 1e-3
    Sw = _cube(rng, z, m)
    T = _cube(rng, z, m)
    tol = flip_tolerance(Sw, T, cube_err=err, base=0.0)
    base = _pearson_maps(Sw, T)[0, 0]
    lo = bf16_round(Sw)
    u = bf16_ulp(Sw)
    amb = np.minimum(np.abs(Sw - (lo + u / 2)), np.abs(Sw - (lo - u / 2))) <= err
    idx = np.argwhere(amb)
    assert len(idx) > 5
    for i in idx[:40]:
        S2 = Sw.copy()
        S2[tuple(i)] += u[tuple(i)]
        assert abs(_pearson_maps(S2, T)[0, 0] - base) <= tol


def _parabola(cm, c0, cp):
    den = cm - 2 * c0 + cp
    return 0.0 if den >= 0 else float(np.clip((cm - cp) / (2 * den), -0.5, 0.5))


@pytest.mark.parametrize("seed", [8, 9, 10])
def test_subpixel_tolerance_covers_map_errors(seed):
    """Every map error of at most e at the three samples moves the parabola
    vertex by at most subpixel_tol(e) on each axis."""
    rng = np.random.default_rng(seed)
    R, e = 4, 1e-3
    P1 = 2 * R + 1
    for _ in range(20):
        vy, vx = rng.uniform(-0.45, 0.45, 2)
        ky, kx = rng.uniform(0.01, 0.2, 2)
        yy, xx = np.mgrid[-R:R + 1, -R:R + 1].astype(np.float64)
        omap = 0.9 - ky * (yy - vy) ** 2 - kx * (xx - vx) ** 2
        tol = subpixel_tol(omap, R, e, base=0.0)
        c = R
        for _ in range(30):
            g = omap + rng.uniform(-e, e, omap.shape)
            if int(np.argmax(g)) != c * P1 + c:
                continue
            dx = _parabola(g[c, c - 1], g[c, c], g[c, c + 1]) - _parabola(omap[c, c - 1], omap[c, c], omap[c, c + 1])
            dy = _parabola(g[c - 1, c], g[c, c], g[c + 1, c]) - _parabola(omap[c - 1, c], omap[c, c], omap[c + 1, c])
            assert max(abs(dx), abs(dy)) <= tol + 1e-12


def _res(dx, dy, ncc, status=None):
    n = len(dx)
    return {"dx": np.asarray(dx), "dy": np.asarray(dy), "ncc": np.asarray(ncc, np.float32),
            "sub_dx": np.zeros(n, np.float32), "sub_dy": np.zeros(n, np.float32),
            "status": np.zeros(n, np.int32) if status is None else np.asarray(status)}


def test_compare_accepts_valid_ties_and_rejects_wrong_offsets():
    R = 1
    omap = np.full((3, 3), 0.2)
    omap[1, 1], omap[1, 2] = 0.9, 0.9 - 1e-4        # a near-tie with (dx, dy) = (1, 0)
    orc = _res([0], [0], [0.9])
    orc.update(margin=np.array([1e-4]), sub_dx=np.zeros(1), sub_dy=np.zeros(1))
    compare(_res([1], [0], [0.9 - 1e-4]), orc, R, oracle_maps=omap[None])      # the other argmax: valid
    with pytest.raises(AssertionError):
        compare(_res([-1], [0], [0.2]), orc, R, oracle_maps=omap[None])        # not an argmax
    orc2 = dict(orc, margin=np.array([0.5]))
    with pytest.raises(AssertionError):
        compare(_res([1], [0], [0.9]), orc2, R, oracle_maps=omap[None])        # clear peak: must match
    with pytest.raises(AssertionError):
        compare(_res([0], [0], [0.9 + 2e-4]), orc2, R, oracle_maps=omap[None])  # NCC beyond 1e-4
    with pytest.raises(AssertionError):
        compare(_res([0], [0], [0.9], status=[2]), orc2, R)                    # status differs


def test_compare_bounds_and_reports_tie_flips(tmp_path, monkeypatch):
    """Near-ties are counted and logged; valid tie flips beyond 1 % of the
    valid points (at least one allowed) fail the comparison."""
    import json
    R, n = 1, 3
    omap = np.full((n, 3, 3), 0.2)
    omap[:, 1, 1], omap[:, 1, 2] = 0.9, 0.9 - 1e-4  # every point a near-tie
    orc = _res([0] * n, [0] * n, [0.9] * n)
    orc.update(margin=np.full(n, 1e-4), sub_dx=np.zeros(n), sub_dy=np.zeros(n))
    log = tmp_path / "ties.jsonl"
    monkeypatch.setenv("SFOC_PARITY_LOG", str(log))
    st = compare(_res([1, 0, 0], [0] * n, [0.9 - 1e-4, 0.9, 0.9]), orc, R, oracle_maps=omap)  # one flip: allowed
    assert st["near_ties"] == 3 and st["tie_flips"] == 1
    rec = json.loads(log.read_text().splitlines()[-1])
    assert rec["near_ties"] == 3 and rec["tie_flips"] == 1
    with pytest.raises(AssertionError, match="tie flips"):
        compare(_res([1, 1, 0], [0] * n, [0.9 - 1e-4, 0.9 - 1e-4, 0.9]), orc, R, oracle_maps=omap)
