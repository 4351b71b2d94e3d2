"""Pins of the RANSAC oracle (Sec. 3.2.3) and of the matching criteria of
Sec. 4.1 (NCM, CMR, RMSE of Eq. 22) against facts fixed by the geometry:
exact recovery of planted models, the exactness of a minimal solve on its
own sample, degenerate samples, the tie rule, the threshold boundary and
closed-form criteria."""
import numpy as np
import pytest

import oracle
from workloads import apply_model, planted_correspondences, ransac_samples


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


@pytest.mark.parametrize("projective", [True, False])
@pytest.mark.parametrize("n,frac,seed", [(60, 0.2, 1), (400, 0.5, 2), (1500, 0.3, 3)])
def test_recovers_planted_model(orc, projective, n, frac, seed):
    src, dst, H0, out = planted_correspondences(seed, n, projective, frac)
    k = 4 if projective else 3
    samp = ransac_samples(seed + 100, n, 600, k)
    r = orc.ransac(src, dst, samp, model=orc.PROJECTIVE if projective else orc.AFFINE)
    assert r["best"] >= 0
    np.testing.assert_array_equal(r["inlier"], ~out)
    assert r["count"] == int((~out).sum())
    # exact data: the least-squares refit reproduces the planted model
    assert np.abs(r["H"] - H0).max() <= 1e-9 * np.abs(H0).max()


def test_noisy_inliers_within_threshold(orc):
    src, dst, H0, out = planted_correspondences(7, 800, True, 0.3, noise=0.3)
    samp = ransac_samples(8, 800, 2000, 4)
    r = orc.ransac(src, dst, samp, tau=1.5)
    # every outlier is >= 20 px off, every inlier within a few noise sigmas
    assert not r["inlier"][out].any()
    assert r["inlier"][~out].mean() > 0.99
    # the refit model maps the source points within the noise of the planted one
    d = np.linalg.norm(apply_model(r["H"], src) - apply_model(H0, src), axis=1)
    assert d.max() < 0.2


@pytest.mark.parametrize("projective", [True, False])
def test_minimal_fit_reproduces_its_sample(orc, projective):
    rng = np.random.default_rng(11)
    src = rng.uniform(0, 1000, (20, 2))
    dst = rng.uniform(0, 1000, (20, 2))   # arbitrary: a minimal sample is always fitted exactly
    k = 4 if projective else 3
    for trial in range(20):
        idx = rng.choice(20, k, replace=False)
        H = orc.ransac_fit(src, dst, idx, model=orc.PROJECTIVE if projective else orc.AFFINE)
        assert H is not None
        assert H[2, 2] == 1.0
        np.testing.assert_allclose(apply_model(H, src[idx]), dst[idx], atol=1e-7)


def test_collinear_sample_is_singular(orc):
    src = np.array([[0, 0], [10, 10], [20, 20], [30, 30], [5, 90.0]])
    dst = src + 3.0
    assert orc.ransac_fit(src, dst, [0, 1, 2, 3]) is None           # four collinear points
    assert orc.ransac_fit(src, dst, [0, 1, 2], model=orc.AFFINE) is None
    assert orc.ransac_fit(src, dst, [0, 1, 4], model=orc.AFFINE) is not None
    r = orc.ransac(src, dst, [[0, 1, 2, 3], [0, 1, 2, 3]])
    assert list(r["scores"]) == [-1, -1] and r["best"] == -1 and r["count"] == 0


def test_ties_go_to_the_lower_index(orc):
    src, dst, H0, out = planted_correspondences(5, 100, True, 0.2)
    inl = np.flatnonzero(~out)
    s = inl[:4]
    r = orc.ransac(src, dst, [s, s[::-1], s], refits=0)
    assert r["scores"][0] == r["scores"][1] == r["scores"][2]
    assert r["best"] == 0


def test_threshold_is_inclusive(orc):
    # an exactly given translation by (7, -3): errors of exactly tau, 0.5 tau and 2 tau
    P = np.array([[1, 0, 7], [0, 1, -3], [0, 0, 1.0]])
    src = np.array([[0, 0], [100, 0], [0, 100], [100, 100], [50, 50], [60, 20], [20, 60.0]])
    dst = src + np.array([7.0, -3.0])
    dst[4, 0] += 1.5
    dst[5, 1] += 0.75
    dst[6, 0] += 3.0
    assert orc.match_quality(P, src, dst, tau=1.5)["ncm"] == 6
    # RANSAC's solved model carries rounding of ~1e-14 px: points a relative
    # 1e-6 inside and outside the radius
    dst[4, 0] = src[4, 0] + 7.0 + 1.5 * (1 - 1e-6)
    dst[6, 0] = src[6, 0] + 7.0 + 1.5 * (1 + 1e-6)
    r = orc.ransac(src, dst, [[0, 1, 2]], model=orc.AFFINE, tau=1.5, refits=0)
    assert list(r["inlier"]) == [True, True, True, True, True, True, False]


def test_invalid_points_are_ignored(orc):
    src, dst, H0, out = planted_correspondences(9, 200, True, 0.3)
    valid = np.ones(200, bool)
    valid[::3] = False
    samp = ransac_samples(10, 200, 500, 4)
    samp = samp[np.all(valid[samp], axis=1)]
    r = orc.ransac(src, dst, samp, valid=valid)
    np.testing.assert_array_equal(r["inlier"], ~out & valid)


def test_match_quality_closed_form(orc):
    P = np.array([[1, 0, 5], [0, 1, -2], [0, 0, 1.0]])
    src = np.arange(20, dtype=float).reshape(10, 2) * 17
    dst = apply_model(P, src)
    dst[:6] += np.array([0.6, 0.8])        # 6 correct matches at exactly 1 px
    dst[6:] += np.array([6.0, 8.0])        # 4 wrong ones at 10 px
    q = orc.match_quality(P, src, dst)
    assert q["ncm"] == 6
    assert q["cmr"] == pytest.approx(0.6, abs=1e-15)
    assert q["rmse"] == pytest.approx(1.0, abs=1e-12)
    # Eq. 22 is a root mean square: correct matches at 0.6 and 1.2 px give sqrt(0.9), not 0.9
    d2 = apply_model(P, src)
    d2[:3] += np.array([0.36, 0.48])
    d2[3:6] += np.array([0.72, 0.96])
    d2[6:] += np.array([6.0, 8.0])
    q = orc.match_quality(P, src, d2)
    assert q["ncm"] == 6 and q["rmse"] == pytest.approx(np.sqrt(0.9), abs=1e-12)
    valid = np.ones(10, bool)
    valid[6:] = False                       # only the correct ones count as matches
    q = orc.match_quality(P, src, dst, valid=valid)
    assert (q["ncm"], q["cmr"]) == (6, 1.0)
