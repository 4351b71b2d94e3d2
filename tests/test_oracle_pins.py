"""Pins of the FP64 oracle against what the paper and mathematics fix.

Nothing here compares the oracle with itself: kernels are checked against
numerical derivatives of the Gaussian of Eq. 1, steering against symmetry
and closed forms, NCC against numpy's Pearson correlation, the FFT /
integral-image rewrite (Eq. 9, 13-16) against Eq. 8, and the complexity
model against the value the paper prints.  Each test names the passage.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if not line:
            continue
        k, v = (s.strip() for s in line.split("=", 1))
        vals[k] = v
    return vals


def gauss(x, y, s):
    """Eq. 1 evaluated at real (x, y)."""
    return np.exp(-(x * x + y * y) / (2 * s * s)) / (2 * math.pi * s * s)


# --------------------------------------------------------------------------
# paper constants
# --------------------------------------------------------------------------

def test_complexity_ratio_matches_paper(orc):
    """Eq. 19 with z=9, m=100, M=200 gives the 0.965% printed after Eq. 19."""
    g = golden()
    r = orc.complexity_ratio(int(g["complexity_z"]), int(g["complexity_m"]), int(g["complexity_m"]),
                             int(g["complexity_M"]), int(g["complexity_M"]))
    assert round(100 * r, 3) == pytest.approx(float(g["complexity_ratio_percent"]), abs=1e-9)
    # and it falls as the template grows (Fig. 5 trend)
    assert orc.complexity_ratio(9, 40, 40, 80, 80) > orc.complexity_ratio(9, 100, 100, 200, 200)


def test_default_params_match_table2(orc):
    g = golden()
    p = orc.params()
    assert [p.scales[i] for i in range(p.n_scales)] == [float(g["sigma1"]), float(g["sigma2"]), float(g["sigma3"])]
    assert p.sigma2 == float(g["sigma4"])
    assert p.n_orient == int(g["n_orient"])
    assert [p.dil[i] for i in range(p.n_dil)] == [int(v) for v in g["dilations"].split(",")]
    assert orc.channels(p) == 12
    # kernel radius ceil(3 sigma)
    assert [orc.radius(s) for s in (0.6, 0.8, 1.0, 1.5)] == [2, 3, 3, 5]


# --------------------------------------------------------------------------
# kernels (Eq. 2, 3, 5) against numerical derivatives of Eq. 1
# --------------------------------------------------------------------------

@pytest.mark.parametrize("sigma", [0.6, 0.8, 1.0, 1.5, 3.0])
def test_first_order_kernels_are_gaussian_derivatives(orc, sigma):
    K = orc.radius(sigma)
    gx, gy = orc.kernel_g1(sigma, K)
    t = np.arange(-K, K + 1, dtype=np.float64)
    X, Y = np.meshgrid(t, t)
    h = 1e-5
    dgx = (gauss(X + h, Y, sigma) - gauss(X - h, Y, sigma)) / (2 * h)
    dgy = (gauss(X, Y + h, sigma) - gauss(X, Y - h, sigma)) / (2 * h)
    scale = np.abs(dgx).max()
    np.testing.assert_allclose(gx, dgx, atol=1e-8 * scale)
    np.testing.assert_allclose(gy, dgy, atol=1e-8 * scale)
    # antisymmetric: taps sum to exactly zero in exact arithmetic
    assert abs(gx.sum()) < 1e-15 and abs(gy.sum()) < 1e-15
    # Eq. 3 is Eq. 2 rotated by 90 degrees
    np.testing.assert_array_equal(gy, gx.T)


@pytest.mark.parametrize("theta", np.linspace(0, math.pi, 7))
def test_first_order_steering_eq4(orc, theta):
    """A derivative of Eq. 1 along (cos t, sin t), sampled directly, equals
    cos t * G^0 + sin t * G^90 (Eq. 4)."""
    s = 1.0
    K = orc.radius(s)
    gx, gy = orc.kernel_g1(s, K)
    t = np.arange(-K, K + 1, dtype=np.float64)
    X, Y = np.meshgrid(t, t)
    h = 1e-5
    c, sn = math.cos(theta), math.sin(theta)
    direct = (gauss(X + h * c, Y + h * sn, s) - gauss(X - h * c, Y - h * sn, s)) / (2 * h)
    np.testing.assert_allclose(c * gx + sn * gy, direct, atol=1e-9)


@pytest.mark.parametrize("sigma", [1.0, 1.5, 2.0])
def test_second_order_kernels(orc, sigma):
    """G_xx, G_yy, G_xy are second derivatives of Eq. 1 (Eq. 5); the zero-sum
    correction only subtracts a per-row (per-column) constant."""
    K = orc.radius(sigma)
    gxx, gyy, gxy = orc.kernel_g2(sigma, K)
    t = np.arange(-K, K + 1, dtype=np.float64)
    X, Y = np.meshgrid(t, t)
    h = 1e-4
    dxx = (gauss(X + h, Y, sigma) - 2 * gauss(X, Y, sigma) + gauss(X - h, Y, sigma)) / h ** 2
    dxy = (gauss(X + h, Y + h, sigma) - gauss(X + h, Y - h, sigma) - gauss(X - h, Y + h, sigma)
           + gauss(X - h, Y - h, sigma)) / (4 * h * h)
    scale = np.abs(dxx).max()
    np.testing.assert_allclose(gxy, dxy, atol=1e-6 * scale)
    diff = gxx - dxx
    # difference is constant along x within each row
    np.testing.assert_allclose(diff, np.repeat(diff[:, :1], diff.shape[1], 1), atol=1e-6 * scale)
    # rows of the corrected kernel sum to zero -> zero response to constants
    np.testing.assert_allclose(gxx.sum(1), 0, atol=1e-15)
    np.testing.assert_allclose(gyy, gxx.T, atol=0)
    assert abs(gxy.sum()) < 1e-15


@pytest.mark.parametrize("theta", np.linspace(0, math.pi, 5))
def test_second_order_freeman_adelson(orc, theta):
    """Directional second derivative at theta equals the k_j(theta)
    interpolation of true rotated bases at 0/60/120 deg (Eq. 5, k_j), and the
    cos^2/sin^2/cross form of the Cartesian bases."""
    s = 1.5
    K = orc.radius(s)
    t = np.arange(-K, K + 1, dtype=np.float64)
    X, Y = np.meshgrid(t, t)
    h = 1e-4

    def d2(a):
        c, sn = math.cos(a), math.sin(a)
        return (gauss(X + h * c, Y + h * sn, s) - 2 * gauss(X, Y, s) + gauss(X - h * c, Y - h * sn, s)) / h ** 2

    thetas = [0.0, math.pi / 3, 2 * math.pi / 3]
    k = [(1 + 2 * math.cos(2 * (theta - tj))) / 3 for tj in thetas]
    interp = sum(kj * d2(tj) for kj, tj in zip(k, thetas))
    np.testing.assert_allclose(interp, d2(theta), atol=1e-6 * np.abs(d2(0)).max())


def test_dilated_kernel(orc):
    for sd, r in [(1.0, 1), (1.0, 2), (1.5, 3)]:
        Kd = orc.radius(sd)
        w = orc.kernel_dilated(sd, Kd, r)
        assert w.shape == (2 * r * Kd + 1,) * 2
        assert abs(w.sum() - 1.0) < 1e-14
        nz = np.argwhere(w != 0)
        assert np.all(nz % r == 0)          # holes between the taps
        assert len(nz) == (2 * Kd + 1) ** 2
        c = r * Kd
        # Gaussian profile: g(1)/g(0) = exp(-1 / 2 sd^2)
        assert w[c, c + r] / w[c, c] == pytest.approx(math.exp(-1 / (2 * sd * sd)), rel=1e-13)


def test_conv2d_is_convolution_with_clamped_borders(orc):
    rng = np.random.default_rng(1)
    img = rng.random((9, 11))
    k = rng.random((5, 5))
    # an impulse returns the kernel itself (convolution, not correlation)
    imp = np.zeros((11, 11)); imp[5, 5] = 1.0
    out = orc.conv2d(imp, k)
    np.testing.assert_allclose(out[3:8, 3:8], k, atol=0)
    # interior agrees with scipy's convolve; borders clamp (scipy 'nearest')
    from scipy.ndimage import convolve
    np.testing.assert_allclose(orc.conv2d(img, k), convolve(img, k, mode="nearest"), atol=1e-13)


# --------------------------------------------------------------------------
# SFOC assembly (Eq. 6, 7 and the dilated smoothing + normalisation text)
# --------------------------------------------------------------------------

def _theta(n):
    return np.arange(n) * math.pi / n


def test_sfoc_ramp_closed_form(orc):
    """On a linear ramp I = a x + b y all first-order responses are constant,
    all second-order ones zero (up to rounding), so with a negligible eps the
    first group is |a cos t_k + b sin t_k| normalised and the second group
    zero (eps=0 would blow rounding noise up to unit length)."""
    a, b = 7.0, -3.0          # integer ramp: exact in float32
    n = 64
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    img = a * xx + b * yy
    p = orc.params(eps=1e-7)
    cube = orc.sfoc_roi(img.astype(np.float32), p, 30, 30, 4, 4).data
    th = _theta(6)
    v = np.abs(a * np.cos(th) + b * np.sin(th))
    v /= np.linalg.norm(v)
    for k in range(6):
        np.testing.assert_allclose(cube[k], v[k], atol=1e-7)
    np.testing.assert_allclose(cube[6:], 0.0, atol=1e-6)


def test_sfoc_rotation_covariance(orc):
    """A 90-degree rotation of the image maps orientation k to k+3 (mod 6) in
    both groups; a transpose maps k to 3-k (mod 6).  Exact for the sampled
    kernels (Eq. 4-7 are steerable; the grid maps to itself)."""
    rng = np.random.default_rng(7)
    img = rng.random((40, 40)).astype(np.float32)
    p = orc.params()
    c0 = orc.sfoc_roi(img, p).data
    c_t = orc.sfoc_roi(np.ascontiguousarray(img.T), p).data
    c_r = orc.sfoc_roi(np.ascontiguousarray(np.rot90(img)), p).data
    for g in (0, 6):
        for k in range(6):
            np.testing.assert_allclose(c_t[g + (3 - k) % 6], c0[g + k].T, atol=1e-12)
            np.testing.assert_allclose(c_r[g + (k + 3) % 6], np.rot90(c0[g + k]), atol=1e-12)


@pytest.mark.parametrize("a,b", [(2.0, 0.1), (-0.5, 1.0), (0.01, -3.0)])
def test_sfoc_affine_invariance(orc, a, b):
    """With eps=0, |.| and zero-sum taps, SFOC(a I + b) = SFOC(I) for a != 0
    (the descriptor is invariant to affine intensity changes, incl. inversion)."""
    rng = np.random.default_rng(3)
    img = rng.random((36, 30))
    p = orc.params(eps=0.0)
    c0 = orc.sfoc_roi(img.astype(np.float32), p).data
    c1 = orc.sfoc_roi((a * img.astype(np.float32).astype(np.float64) + b).astype(np.float32), p).data
    # float32 rounding of the transformed input is the only difference
    np.testing.assert_allclose(c1, c0, atol=2e-4)
    # exact version with an exactly representable map
    img2 = np.round(rng.random((30, 30)) * 64).astype(np.float32)
    d0 = orc.sfoc_roi(img2, p).data
    d1 = orc.sfoc_roi((-4.0 * img2 + 1024.0).astype(np.float32), p).data
    np.testing.assert_allclose(d1, d0, atol=1e-12)


def test_sfoc_constant_image_is_zero(orc):
    img = np.full((25, 25), 0.37, np.float32)
    cube = orc.sfoc_roi(img, orc.params()).data
    # taps sum to zero up to double rounding; eps keeps the result tiny
    np.testing.assert_allclose(cube, 0.0, atol=1e-12)


def test_sfoc_x_only_image_reduces_to_1d(orc):
    """An image varying only along x turns every 2-D convolution into a 1-D
    convolution with the kernel's column sums, so the cube can be rebuilt in
    1-D with numpy: pins scale summation, |.|, the group smoothing STDs, the
    dilation rates, the normalisation and the channel order."""
    rng = np.random.default_rng(11)
    W = 96
    prof = np.cumsum(rng.standard_normal(W)) * 0.05
    prof[40:44] += 1.0
    img = np.tile(prof, (48, 1)).astype(np.float32)
    p = orc.params()
    cube = orc.sfoc_roi(img, p, 20, 0, 4, W).data[:, 0, :]

    def conv1(f, k):
        K = (len(k) - 1) // 2
        fp = np.pad(f, K, mode="edge")
        return np.array([sum(k[q + K] * fp[x - q + K] for q in range(-K, K + 1)) for x in range(len(f))])

    x = prof.astype(np.float32).astype(np.float64)
    th = _theta(6)
    F1 = np.zeros((6, W))
    for s in (0.6, 0.8, 1.0):
        K = orc.radius(s)
        gx, gy = orc.kernel_g1(s, K)
        ix = conv1(x, gx.sum(0))
        iy = conv1(x, gy.sum(0))
        assert np.abs(iy).max() < 1e-14
        for k in range(6):
            F1[k] += np.abs(math.cos(th[k]) * ix + math.sin(th[k]) * iy)
    K2 = orc.radius(1.5)
    gxx, gyy, gxy = orc.kernel_g2(1.5, K2)
    ixx = conv1(x, gxx.sum(0))
    F2 = np.array([np.abs(math.cos(t) ** 2 * ixx) for t in th])

    def smooth(F, sd):
        Kd = orc.radius(sd)
        out = np.zeros_like(F)
        for r in (1, 2, 3):
            w = orc.kernel_dilated(sd, Kd, r).sum(0)
            out += np.array([conv1(f, w) for f in F])
        return out

    D1 = smooth(F1, 1.0)
    D2 = smooth(F2, 1.5)
    D1 = D1 / (np.linalg.norm(D1, axis=0) + 1e-3)
    D2 = D2 / (np.linalg.norm(D2, axis=0) + 1e-3)
    np.testing.assert_allclose(cube[:6], D1, atol=1e-12)
    np.testing.assert_allclose(cube[6:], D2, atol=1e-12)


def test_sfoc_roi_equals_full(orc):
    rng = np.random.default_rng(5)
    img = rng.random((50, 45)).astype(np.float32)
    p = orc.params()
    full = orc.sfoc_roi(img, p).data
    part = orc.sfoc_roi(img, p, 3, 30, 20, 15).data
    np.testing.assert_allclose(part, full[:, 3:23, 30:45], atol=0)


def test_first_order_only_variant(orc):
    rng = np.random.default_rng(9)
    img = rng.random((30, 30)).astype(np.float32)
    p = orc.params(first_order_only=True)
    c = orc.sfoc_roi(img, p).data
    assert c.shape[0] == 6
    full = orc.sfoc_roi(img, orc.params()).data
    np.testing.assert_allclose(c, full[:6], atol=0)



@pytest.mark.parametrize("a,b,c", [(1, 3, -2), (-2, 1, 1), (0, 2, 0)])
def test_second_order_channel_is_the_directional_second_derivative(orc, a, b, c):
    """Eq. 7 read with x right and y down: second-order channel theta is the
    second derivative along (cos theta, -sin theta).  On a quadratic image
    I = a x^2 + b x y + c y^2 that derivative is exact from the image itself,
    2a cos^2 - 2b cos sin + 2c sin^2, with no kernel involved.  The sampled,
    truncated kernels reproduce d^2/dx^2 and d^2/dx dy of a quadratic to
    within 1.8 % and 0.7 % (their second moments), so each term may be off
    by 2 %; a flipped or halved cross term is off by far more.  Read
    unsmoothed (sigma_d = 0), signed (rectify off) and before the group
    normalisation (eps = 1e30: an exact division by 1e30)."""
    n = 31
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64) - 15          # x right, y down, origin at the centre
    img = (a * xx * xx + b * xx * yy + c * yy * yy).astype(np.float32)   # integers: exact in FP32
    D = orc.sfoc_roi(img, orc.params(sigma_d1=0.0, sigma_d2=0.0, eps=1e30, rectify=False), 15, 15, 1, 1).data
    D = D[:, 0, 0] * 1e30
    for k, th in enumerate(_theta(6)):
        cs, sn = math.cos(th), math.sin(th)
        terms = (2 * a * cs * cs, -2 * b * cs * sn, 2 * c * sn * sn)
        assert D[6 + k] == pytest.approx(sum(terms), abs=0.02 * sum(abs(t) for t in terms) + 1e-9), k

def _pre_norm(orc, img, **kw):
    """The input D of the group normalisation: with eps = 1e30 the division
    by ||D|| + eps is an exact division by 1e30 (||D|| is far below the
    spacing of doubles near 1e30), so the cube times 1e30 returns D to
    within two roundings."""
    return orc.sfoc_roi(img, orc.params(eps=1e30, **kw)).data * 1e30


def _dilated_smooth(F, sd, rates):
    """Parallel dilated Gaussian of Sec. 2.1 through scipy: taps
    exp(-t^2 / 2 sd^2) / sum over |t| <= ceil(3 sd), spread to spacing r,
    applied separably with edge replication, summed over r."""
    from scipy.ndimage import correlate1d
    K = math.ceil(3 * sd - 1e-9)
    t = np.arange(-K, K + 1)
    g = np.exp(-t * t / (2 * sd * sd))
    g /= g.sum()
    out = np.zeros_like(F)
    for r in rates:
        w = np.zeros(2 * r * K + 1)
        w[::r] = g
        out += correlate1d(correlate1d(F, w, axis=0, mode="nearest"), w, axis=1, mode="nearest")
    return out


def test_no_smoothing_variant_feeds_the_smoothing(orc):
    """sigma_d = 0 switches the smoothing off (the descriptor without
    Gaussian convolution of Fig. 3 (d), Sec. 2.1): its pre-normalisation
    planes are the steered channels F, and scipy's Gaussian filters of those
    planes reproduce the paper's parallel dilated smoothing (Fig. 3 (f)) and
    the plain Gaussian of Fig. 3 (e) (one rate, r = 1).  A wrong offset or
    channel in the unsmoothed branch, or a wrong rate, STD or border in the
    smoothed one, breaks the agreement."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(21)
    from workloads import optical_like
    img = optical_like(rng, 48, 61)
    F = _pre_norm(orc, img, sigma_d1=0.0, sigma_d2=0.0)
    assert F.shape == (12, 48, 61) and np.abs(F).max() > 1e-2
    D = _pre_norm(orc, img)
    Dg = _pre_norm(orc, img, dil=(1,))
    for c in range(12):
        sd = 1.0 if c < 6 else 1.5      # group STDs of the defaults
        scale = np.abs(D[c]).max()
        np.testing.assert_allclose(D[c], _dilated_smooth(F[c], sd, (1, 2, 3)), atol=1e-13 * scale + 1e-300)
        np.testing.assert_allclose(Dg[c], gaussian_filter(F[c], sd, mode="nearest", truncate=3.0),
                                   atol=1e-13 * scale + 1e-300)
    # one group smoothed, the other not
    Dm = _pre_norm(orc, img, sigma_d1=0.0)
    np.testing.assert_allclose(Dm[:6], F[:6], atol=0)
    np.testing.assert_allclose(Dm[6:], D[6:], atol=0)


def test_no_smoothing_is_the_narrow_gaussian_limit(orc):
    """As sigma_d shrinks the taps off the centre vanish (exp(-200) at
    sigma_d = 0.05); with eps = 0 the sum over three rates only scales the
    group, which the normalisation removes, so sigma_d = 0 is the limit."""
    rng = np.random.default_rng(22)
    img = rng.random((30, 37)).astype(np.float32)
    c0 = orc.sfoc_roi(img, orc.params(eps=0.0, sigma_d1=0.0, sigma_d2=0.0)).data
    c1 = orc.sfoc_roi(img, orc.params(eps=0.0, sigma_d1=0.05, sigma_d2=0.05)).data
    np.testing.assert_allclose(c0, c1, atol=1e-13)
    with pytest.raises(RuntimeError):
        orc.sfoc_roi(img, orc.params(sigma_d1=-1.0))

# --------------------------------------------------------------------------
# NCC (Eq. 8), its rewrite (Eq. 9, 13-16), argmax and sub-pixel
# --------------------------------------------------------------------------

def _cube(data, H=None, W=None, y0=0, x0=0):
    import oracle
    z, h, w = data.shape
    return oracle.CubeROI(np.ascontiguousarray(data, np.float64), H or h, W or w, y0, x0)


def test_ncc_equals_pearson(orc):
    """Eq. 8 is the Pearson correlation of the flattened m x m x z windows."""
    rng = np.random.default_rng(2)
    z, H, W, m, R = 3, 30, 31, 7, 4
    ref = rng.random((z, H, W))
    sen = rng.random((z, H, W))
    pts = np.array([[12, 13], [15, 16]], np.int32)
    out = orc.match(_cube(ref), _cube(sen), pts, m, R, want_maps=True)
    h = (m - 1) // 2
    for k, (px, py) in enumerate(pts):
        T = sen[:, py - h:py - h + m, px - h:px - h + m].ravel()
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                S = ref[:, py - h + dy:py - h + dy + m, px - h + dx:px - h + dx + m].ravel()
                assert out["maps"][k, dy + R, dx + R] == pytest.approx(np.corrcoef(S, T)[0, 1], abs=1e-13)


@pytest.mark.parametrize("z,m,R", [(2, 3, 1), (1, 4, 2), (2, 5, 2)])
def test_eq9_fft_integral_equals_eq8(orc, z, m, R):
    """Eq. 9 with R_ST from the DFT of Eq. 13 and R_S, R_SS from integral
    images (Eq. 14-16) equals Eq. 8 on tiny inputs."""
    rng = np.random.default_rng(z * 100 + m * 10 + R)
    M = m + 2 * R
    S = rng.random((z, M, M))
    T = rng.random((z, m, m))
    a = orc.ncc_eq9_dft(S, T, R)
    b = orc.ncc_eq9_dft(S, T, R, L=M + 3)        # more padding, same result
    # Eq. 8 through the matcher: put the window in a "reference" and the
    # template in a "sensed" cube at the same place
    H = M
    ref = S
    sen = np.zeros((z, H, H)); sen[:, R:R + m, R:R + m] = T
    h = (m - 1) // 2 if m % 2 else m // 2
    pts = np.array([[R + h, R + h]], np.int32)
    c = orc.match(_cube(ref), _cube(sen), pts, m, R, want_maps=True)["maps"][0]
    np.testing.assert_allclose(a, c, atol=1e-11)
    np.testing.assert_allclose(b, c, atol=1e-11)
    # and numpy's FFT gives the same R_ST as the naive DFT path implies
    Lf = 2 * M
    acc = np.zeros((Lf, Lf), complex)
    for ch in range(z):
        acc += np.fft.fft2(S[ch], (Lf, Lf)) * np.conj(np.fft.fft2(T[ch], (Lf, Lf)))
    rst = np.real(np.fft.ifft2(acc))[:2 * R + 1, :2 * R + 1]
    direct = np.array([[sum((S[ch, dy:dy + m, dx:dx + m] * T[ch]).sum() for ch in range(z))
                        for dx in range(2 * R + 1)] for dy in range(2 * R + 1)])
    np.testing.assert_allclose(rst, direct, atol=1e-10)


def test_integral_image_rect_sums(orc):
    """Eq. 16 on the exclusive prefix equals brute-force sums (exact on
    integer data)."""
    rng = np.random.default_rng(4)
    g = rng.integers(-50, 50, (13, 17)).astype(np.float64)
    P = orc.integral(g)
    assert P.shape == (14, 18)
    for _ in range(200):
        y0, y1 = sorted(rng.integers(0, 14, 2))
        x0, x1 = sorted(rng.integers(0, 18, 2))
        assert orc.rect_sum(P, y0, x0, y1, x1) == g[y0:y1, x0:x1].sum()


def test_ncc_self_template_is_one(orc):
    """A template cut from the same image scores NCC = 1 at d = 0 and < 1
    elsewhere (Eq. 8)."""
    rng = np.random.default_rng(8)
    c = rng.random((4, 40, 40))
    pts = np.array([[20, 20], [17, 22]], np.int32)
    out = orc.match(_cube(c), _cube(c), pts, 9, 5, want_maps=True)
    assert np.all(out["dx"] == 0) and np.all(out["dy"] == 0)
    np.testing.assert_allclose(out["ncc"], 1.0, atol=1e-14)
    for k in range(2):
        mp = out["maps"][k].copy()
        mp[5, 5] = -2
        assert mp.max() < 1.0


@pytest.mark.parametrize("a,b", [(3.0, 1.0), (0.2, -5.0), (-1.5, 0.3)])
def test_ncc_affine_invariance(orc, a, b):
    """NCC(a T + b, S) = sign(a) NCC(T, S) (Eq. 8)."""
    rng = np.random.default_rng(6)
    ref = rng.random((3, 30, 30))
    sen = rng.random((3, 30, 30))
    pts = np.array([[15, 15]], np.int32)
    m0 = orc.match(_cube(ref), _cube(sen), pts, 7, 3, want_maps=True)["maps"][0]
    m1 = orc.match(_cube(ref), _cube(a * sen + b), pts, 7, 3, want_maps=True)["maps"][0]
    np.testing.assert_allclose(m1, np.sign(a) * m0, atol=1e-12)


def test_ncc_channel_permutation_invariance(orc):
    rng = np.random.default_rng(12)
    ref = rng.random((6, 30, 30))
    sen = rng.random((6, 30, 30))
    perm = [3, 1, 5, 0, 2, 4]
    pts = np.array([[14, 15]], np.int32)
    a = orc.match(_cube(ref), _cube(sen), pts, 7, 3, want_maps=True)["maps"]
    b = orc.match(_cube(ref[perm]), _cube(sen[perm]), pts, 7, 3, want_maps=True)["maps"]
    np.testing.assert_allclose(a, b, atol=1e-13)


def test_planted_shift_recovered_exactly(orc):
    """Sensed = affine map of the reference shifted by s: SFOC is invariant
    (eps=0), so NCC = 1 exactly at d = -s away from the borders."""
    from workloads import optical_like, shift_image
    rng = np.random.default_rng(21)
    ref = optical_like(rng, 96, 96, 6, 4)
    sx, sy = 3, -2
    sen = (shift_image(ref, sx, sy) * np.float32(-2.0) + np.float32(3.0)).astype(np.float32)
    p = orc.params(eps=0.0)
    out = orc.match_pair(ref, sen, np.array([[48, 48], [45, 50]], np.int32), 21, 5, p, roi=False)
    assert np.all(out["dx"] == -sx) and np.all(out["dy"] == -sy)
    np.testing.assert_allclose(out["ncc"], 1.0, atol=1e-5)


def test_parabola_vertex(orc):
    """A quadratic NCC surface with a known vertex: the per-axis 3-point
    parabola returns the vertex exactly."""
    R = 4
    vy, vx = 1.3, -0.2
    d = np.arange(-R, R + 1, dtype=np.float64)
    DY, DX = np.meshgrid(d, d, indexing="ij")
    mp = 0.9 - 0.02 * (DX - vx) ** 2 - 0.03 * (DY - vy) ** 2
    r = orc.pick(mp)
    assert (r["dx"], r["dy"]) == (0, 1)
    assert r["sub_dx"] == pytest.approx(vx, abs=1e-12)
    assert r["sub_dy"] == pytest.approx(vy, abs=1e-12)
    assert r["status"] == 0
    # clamp and non-negative curvature
    assert orc.parabola(0.0, 1.0, 2.0) == 0.0
    assert orc.parabola(0.0, 0.0, 0.0) == 0.0
    assert abs(orc.parabola(0.99, 1.0, 0.0)) <= 0.5
    # vertices inside the clamp are returned as they are, outside it at +-0.5
    for v, want in ((0.45, 0.45), (-0.45, -0.45), (0.7, 0.5), (-0.9, -0.5)):
        f = [-(x - v) ** 2 for x in (-1.0, 0.0, 1.0)]
        assert orc.parabola(*f) == pytest.approx(want, abs=1e-12)


def test_argmax_tiebreak_and_edges(orc):
    R = 2
    mp = np.zeros((5, 5))
    mp[3, 1] = mp[1, 4] = mp[1, 2] = 0.8
    r = orc.pick(mp)
    assert (r["dy"], r["dx"]) == (-1, 0)       # smallest dy, then smallest dx
    assert r["status"] == 0 and r["margin"] == 0.0
    mp2 = np.zeros((5, 5)); mp2[0, 2] = 0.7
    r2 = orc.pick(mp2)
    assert (r2["dy"], r2["dx"]) == (-2, 0) and r2["status"] == 3   # PEAK_ON_EDGE
    assert r2["sub_dy"] == -2.0
    mp3 = np.zeros((5, 5)); mp3[2, 2] = np.nan; mp3[1, 1] = 0.2
    r3 = orc.pick(mp3)
    assert (r3["dy"], r3["dx"]) == (-1, -1) and r3["status"] == 4


def test_status_out_of_bounds_and_flat(orc):
    rng = np.random.default_rng(13)
    ref = rng.random((2, 20, 20))
    sen = rng.random((2, 20, 20))
    sen[:, 3:10, 10:17] = 0.5
    pts = np.array([[3, 10], [13, 3], [10, 10], [16, 10]], np.int32)
    out = orc.match(_cube(ref), _cube(sen), pts, 7, 3)
    assert list(out["status"][:2]) == [1, 1]
    assert out["status"][2] in (0, 3)
    assert out["status"][3] == 1
    out2 = orc.match(_cube(ref), _cube(sen), np.array([[13, 6]], np.int32), 7, 3)
    assert out2["status"][0] == 2                # template is constant
    # the flatness threshold (a reading: variance <= 1e-6 per value): a
    # checkerboard of 1e-5 per value is texture, one of 5e-7 is flat
    cb = np.where(np.add.outer(np.arange(7), np.arange(7)) % 2 == 0, 1.0, -1.0)
    for var, flat in ((1e-5, False), (5e-7, True)):
        s2 = sen.copy()
        s2[:, 3:10, 10:17] = 0.5 + np.sqrt(var) * cb
        st = orc.match(_cube(ref), _cube(s2), np.array([[13, 6]], np.int32), 7, 3)["status"][0]
        assert (st == 2) == flat, (var, st)


def test_even_template_centering(orc):
    assert orc.template_half(80) == 40 and orc.template_half(81) == 40 and orc.template_half(100) == 50
    rng = np.random.default_rng(14)
    c = rng.random((2, 30, 30))
    # even m: template rows p-4 .. p+3; a self-match still peaks at d=0
    out = orc.match(_cube(c), _cube(c), np.array([[15, 15]], np.int32), 8, 3)
    assert (out["dx"][0], out["dy"][0]) == (0, 0)
