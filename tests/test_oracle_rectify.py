"""Pins of the rectification oracle (Sec. 3.2.3: the sensed image resampled
into the reference frame by bilinear interpolation): the identity model
copies, integer translations shift exactly, half-pixel translations average
neighbours, linear ramps are reproduced exactly by bilinear interpolation
under any affine model, and positions outside the image take the fill."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def orc():
    oracle.build()
    return oracle


def test_identity_copies(orc):
    img = np.random.default_rng(1).random((37, 53)).astype(np.float32)
    assert np.array_equal(orc.rectify(img, np.eye(3)), img)


def test_integer_translation_shifts(orc):
    img = np.random.default_rng(2).random((40, 50)).astype(np.float32)
    T = np.array([[1, 0, 5], [0, 1, -3], [0, 0, 1.0]])      # sensed (u, v) -> reference (u + 5, v - 3)
    out = orc.rectify(img, T, fill=-1.0)
    assert np.array_equal(out[0:37, 5:50], img[3:40, 0:45])
    assert (out[37:, :] == -1).all() and (out[:, :5] == -1).all()


def test_half_pixel_shift_averages(orc):
    img = np.random.default_rng(3).random((20, 30)).astype(np.float32)
    T = np.array([[1, 0, -0.5], [0, 1, 0], [0, 0, 1.0]])     # output x samples u = x + 0.5
    out = orc.rectify(img, T)
    want = ((img[:, :-1].astype(np.float64) + img[:, 1:]) / 2).astype(np.float32)
    assert np.array_equal(out[:, :-1], want)


def test_linear_ramp_is_exact_under_affine(orc):
    yy, xx = np.mgrid[0:64, 0:80]
    img = (0.01 * xx + 0.02 * yy + 0.1).astype(np.float32)
    A = np.array([[0.98, 0.05, 3.2], [-0.04, 1.01, -2.7], [0, 0, 1.0]])
    out = orc.rectify(img, A)
    Ai = np.linalg.inv(A)
    u = Ai[0, 0] * xx + Ai[0, 1] * yy + Ai[0, 2]
    v = Ai[1, 0] * xx + Ai[1, 1] * yy + Ai[1, 2]
    inside = (u >= 0) & (v >= 0) & (u <= 79) & (v <= 63)
    ramp = 0.01 * u + 0.02 * v + 0.1
    assert np.abs(out[inside] - ramp[inside]).max() < 1e-5      # float rounding of the stored ramp only
    assert inside.mean() > 0.8


def test_singular_model(orc):
    with pytest.raises(ValueError):
        orc.rectify(np.zeros((5, 5), np.float32), np.zeros((3, 3)))
