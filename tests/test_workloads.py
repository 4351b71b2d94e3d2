"""The seeded generators are deterministic and produce the workload shapes."""
import numpy as np

from workloads import inverting_pair_512, tiny_pair, template_half, margin_for


def test_inverting_pair_512_deterministic_and_shaped():
    a = inverting_pair_512()
    b = inverting_pair_512()
    np.testing.assert_array_equal(a.ref, b.ref)
    np.testing.assert_array_equal(a.sen, b.sen)
    np.testing.assert_array_equal(a.points, b.points)
    assert a.ref.shape == (512, 512) and a.ref.dtype == np.float32
    assert a.ref.flags.c_contiguous and a.sen.flags.c_contiguous
    assert a.points.shape == (100, 2)
    assert 0.0 <= a.ref.min() and a.ref.max() <= 1.0
    sx, sy = a.meta["shift"]
    assert -8 <= sx <= 8 and -8 <= sy <= 8
    lo, hi = margin_for(a.m, a.R)
    assert np.all(a.points >= lo) and np.all(a.points < 512 - hi)


def test_tiny_pair_and_half():
    p = tiny_pair(3, 70, 83, 9, 4, 12)
    assert p.ref.shape == (70, 83)
    assert len(p.points) <= 12
    assert template_half(9) == 4 and template_half(10) == 5


def test_noise_series_statistics():
    """Sec. 4.3 noise: Gaussian of variance v, speckle n * I with n of
    variance v; v = 0 is the identity.  Checked on a mid-grey image so that
    clipping to [0, 1] stays negligible."""
    from workloads import add_noise
    img = np.full((400, 500), 0.5, np.float32)
    rng = np.random.default_rng(0)
    assert np.array_equal(add_noise(rng, img, "gaussian", 0.0), img)
    g = add_noise(rng, img, "gaussian", 0.004) - img
    assert abs(g.mean()) < 1e-3 and abs(g.var() - 0.004) < 2e-4
    sp = add_noise(rng, img, "speckle", 0.04) / img - 1.0
    assert abs(sp.mean()) < 2e-3 and abs(sp.var() - 0.04) < 2e-3
    assert np.abs(sp).max() <= np.sqrt(3 * 0.04) + 1e-6
    assert add_noise(rng, np.ones((50, 50), np.float32), "gaussian", 0.01).max() <= 1.0


def _recovered(pair, k, seed=0):
    """How many of k seeded points the FP64 oracle matches within 1.5 px of
    the generator's truth (Sec. 4.1's correct-match radius), and how many
    within 1.5 px of its negation (a sign error in the truth)."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pair.points), k, replace=False))
    o = oracle.match_pair(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R)
    ok = o["status"] == 0
    off = np.stack([o["sub_dx"], o["sub_dy"]], 1)
    t = pair.truth[idx]
    return (int((ok & (np.linalg.norm(off - t, axis=1) <= 1.5)).sum()),
            int((ok & (np.linalg.norm(off + t, axis=1) <= 1.5) & (np.linalg.norm(t, axis=1) > 3)).sum()))


def test_planted_truth_is_what_the_oracle_finds():
    """The generators' ground truth (the offset d with sensed(p) showing the
    reference at p + d) agrees with what the oracle's matching finds on
    reduced versions of the workloads: the inverting 512^2 pair, the SAR-like
    pair's block shift field, and the per-block affine field of the 10000^2
    pair with its speckle turned off (L = 1 speckle defeats most matches at
    any template size, which is the workload's purpose, not the truth's)."""
    from workloads import inverting_pair_512, sar_pair_2048, speckle_pair_10000
    good, flipped = _recovered(inverting_pair_512(), 8)
    assert good >= 7 and flipped == 0
    good, flipped = _recovered(sar_pair_2048(seed=2100, H=1024, W=1024, grid=8, n_points=64, block=256), 10)
    assert good >= 4 and flipped == 0
    good, flipped = _recovered(speckle_pair_10000(seed=5100, H=1024, W=1024, n_points=36, looks=10 ** 6), 6)
    assert good >= 4 and flipped == 0
