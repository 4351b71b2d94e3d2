"""Seeded synthetic multimodal image pairs and interest points.

This module only fabricates inputs.  It holds none of the arithmetic of the
matching method itself (no steerable filters, no smoothing kernels of the
descriptor, no correlation): images are value noise plus drawn shapes, the
sensed image is a radiometric remap of a shifted or warped copy, and the
interest points come from a simple block-wise gradient / Harris detector.
Both the oracle and the GPU path consume the arrays made here.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64), so a
seed fixes every pixel.  Images are float32 in [0, 1] unless stated.

Workload shapes follow the paper's experiments: 512-1501 px multimodal pairs
(Table 1), template windows of 80-100 px and search windows of 200 px
(Sec. 4.1, Table 4), optical/SAR pairs with speckle (Sec. 5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# image primitives
# --------------------------------------------------------------------------


def _fade(t):
    return t * t * (3.0 - 2.0 * t)


def value_noise(rng, H, W, cell, dtype=np.float32):
    """One octave of value noise: a random lattice with spacing ``cell`` px,
    interpolated with a C1 fade.  Cheap (O(HW)) at any size."""
    gh = H // cell + 2
    gw = W // cell + 2
    lat = rng.random((gh, gw), dtype=np.float32)
    ys = np.arange(H, dtype=np.float32) / cell
    xs = np.arange(W, dtype=np.float32) / cell
    y0 = ys.astype(np.int64)
    x0 = xs.astype(np.int64)
    ty = _fade(ys - y0).astype(dtype)[:, None]
    tx = _fade(xs - x0).astype(dtype)[None, :]
    a = lat[y0][:, x0]
    b = lat[y0][:, x0 + 1]
    c = lat[y0 + 1][:, x0]
    d = lat[y0 + 1][:, x0 + 1]
    top = a + (b - a) * tx
    bot = c + (d - c) * tx
    return (top + (bot - top) * ty).astype(dtype)


def multi_octave_noise(rng, H, W, cells=(64, 32, 16, 8, 4, 2), decay=0.6):
    img = np.zeros((H, W), np.float32)
    amp = 1.0
    for c in cells:
        img += np.float32(amp) * value_noise(rng, H, W, c)
        amp *= decay
    return img


def draw_rects(img, rng, n, min_side=8, max_side=None):
    H, W = img.shape
    if max_side is None:
        max_side = max(min_side + 1, min(H, W) // 6)
    for _ in range(n):
        h = int(rng.integers(min_side, max_side))
        w = int(rng.integers(min_side, max_side))
        y = int(rng.integers(0, max(1, H - h)))
        x = int(rng.integers(0, max(1, W - w)))
        img[y:y + h, x:x + w] += np.float32(rng.uniform(-1.0, 1.0))
    return img


def draw_lines(img, rng, n, max_width=3):
    H, W = img.shape
    for _ in range(n):
        y0, y1 = rng.uniform(0, H - 1, 2)
        x0, x1 = rng.uniform(0, W - 1, 2)
        width = int(rng.integers(1, max_width + 1))
        val = np.float32(rng.uniform(-1.0, 1.0))
        L = int(math.hypot(y1 - y0, x1 - x0)) + 1
        t = np.linspace(0.0, 1.0, 2 * L + 1)
        ys = np.round(y0 + (y1 - y0) * t).astype(np.int64)
        xs = np.round(x0 + (x1 - x0) * t).astype(np.int64)
        for oy in range(width):
            for ox in range(width):
                yy = np.clip(ys + oy, 0, H - 1)
                xx = np.clip(xs + ox, 0, W - 1)
                img[yy, xx] = img[yy, xx] * np.float32(0.3) + val
    return img


def scale01(img):
    lo = float(img.min())
    hi = float(img.max())
    if hi <= lo:
        return np.zeros_like(img, dtype=np.float32)
    return ((img - lo) / (hi - lo)).astype(np.float32)


def optical_like(rng, H, W, n_rects=None, n_lines=None):
    """Reference image: multi-octave value noise + rectangles (fields,
    buildings) + lines (roads), scaled to [0, 1]."""
    area = H * W / (512.0 * 512.0)
    if n_rects is None:
        n_rects = int(30 * area)
    if n_lines is None:
        n_lines = int(20 * area)
    img = multi_octave_noise(rng, H, W)
    img *= np.float32(0.5)
    draw_rects(img, rng, n_rects)
    draw_lines(img, rng, n_lines)
    return scale01(img)


# --------------------------------------------------------------------------
# geometric and radiometric differences
# --------------------------------------------------------------------------


def shift_image(img, sx, sy):
    """sen[y, x] = img[clamp(y - sy), clamp(x - sx)] (integer shift)."""
    H, W = img.shape
    ys = np.clip(np.arange(H) - sy, 0, H - 1)
    xs = np.clip(np.arange(W) - sx, 0, W - 1)
    return np.ascontiguousarray(img[ys][:, xs])


def shift_field_image(img, block, offsets):
    """Piecewise-constant shift: the sensed pixel (y, x) in block
    (y // block, x // block) takes img at (y - sy, x - sx) of that block."""
    H, W = img.shape
    out = np.empty_like(img)
    nby, nbx = offsets.shape[:2]
    for by in range(nby):
        for bx in range(nbx):
            y0, y1 = by * block, min(H, (by + 1) * block)
            x0, x1 = bx * block, min(W, (bx + 1) * block)
            if y0 >= H or x0 >= W:
                continue
            sx, sy = int(offsets[by, bx, 0]), int(offsets[by, bx, 1])
            ys = np.clip(np.arange(y0, y1) - sy, 0, H - 1)
            xs = np.clip(np.arange(x0, x1) - sx, 0, W - 1)
            out[y0:y1, x0:x1] = img[ys][:, xs]
    return out


def bilinear_sample(img, yy, xx):
    """Sample img at float coordinates with edge clamping."""
    H, W = img.shape
    yy = np.clip(yy, 0.0, H - 1.0)
    xx = np.clip(xx, 0.0, W - 1.0)
    y0 = np.minimum(np.floor(yy).astype(np.int64), H - 2 if H > 1 else 0)
    x0 = np.minimum(np.floor(xx).astype(np.int64), W - 2 if W > 1 else 0)
    fy = (yy - y0).astype(np.float32)
    fx = (xx - x0).astype(np.float32)
    y1 = np.minimum(y0 + 1, H - 1)
    x1 = np.minimum(x0 + 1, W - 1)
    a = img[y0, x0]
    b = img[y0, x1]
    c = img[y1, x0]
    d = img[y1, x1]
    top = a + (b - a) * fx
    bot = c + (d - c) * fx
    return top + (bot - top) * fy


def piecewise_inverting_map(rng):
    """Monotone increasing up to a random knot, decreasing after it."""
    k = float(rng.uniform(0.4, 0.8))
    b = float(rng.uniform(0.0, 0.5))

    def f(v):
        v = v.astype(np.float32)
        up = v / np.float32(k)
        down = np.float32(1.0) - np.float32(1.0 - b) * (v - np.float32(k)) / np.float32(1.0 - k)
        return np.where(v <= k, up, down).astype(np.float32)

    return f, (k, b)


def gamma_speckle(rng, shape, looks):
    """Multiplicative speckle with unit mean: Gamma(shape=L, scale=1/L)."""
    return rng.gamma(looks, 1.0 / looks, size=shape).astype(np.float32)


def radiometric(rng, img, kind):
    """One of the mixed batch's maps: linear, gamma, inverted, speckled."""
    if kind == "linear":
        a = rng.uniform(0.5, 1.5)
        b = rng.uniform(-0.2, 0.2)
        return scale01((img * np.float32(a) + np.float32(b)).astype(np.float32))
    if kind == "gamma":
        g = rng.uniform(0.4, 2.5)
        return scale01(np.power(np.maximum(img, 0.0), np.float32(g)).astype(np.float32))
    if kind == "inverted":
        return scale01((np.float32(1.0) - img).astype(np.float32))
    if kind == "speckled":
        return scale01(img * gamma_speckle(rng, img.shape, 4))
    raise ValueError(kind)


def add_noise(rng, img, kind, v):
    """The noise series of Sec. 4.3 on a [0, 1] image: 'gaussian' adds white
    noise of mean 0 and variance v; 'speckle' adds n * I with n uniform of
    mean 0 and variance v (half-width sqrt(3 v)).  The result is clipped to
    [0, 1]; v = 0 returns the image unchanged."""
    img = np.asarray(img, np.float32)
    if v == 0:
        return img.copy()
    if kind == "gaussian":
        n = rng.normal(0.0, math.sqrt(v), img.shape).astype(np.float32)
        out = img + n
    elif kind == "speckle":
        a = math.sqrt(3.0 * v)
        n = rng.uniform(-a, a, img.shape).astype(np.float32)
        out = img + n * img
    else:
        raise ValueError(kind)
    return np.clip(out, 0.0, 1.0).astype(np.float32)

# --------------------------------------------------------------------------
# interest points (harness, not the method)
# --------------------------------------------------------------------------


def _grad_mag(img):
    gy = np.zeros_like(img)
    gx = np.zeros_like(img)
    gy[1:-1] = img[2:] - img[:-2]
    gx[:, 1:-1] = img[:, 2:] - img[:, :-2]
    return gx, gy


def _box3(a):
    p = np.pad(a, 1, mode="edge")
    s = np.zeros_like(a)
    for dy in range(3):
        for dx in range(3):
            s += p[dy:dy + a.shape[0], dx:dx + a.shape[1]]
    return s


def block_points(img, grid_y, grid_x, margin_y, margin_x, score="grad", ref_shape=None):
    """One interest point per grid cell: the maximum of a score inside the
    cell, restricted to [margin, size - margin).  ``score`` is 'grad'
    (squared gradient magnitude) or 'harris'.  Returns int32 (n, 2) as
    (x, y) in row-major cell order; empty cells are skipped."""
    H, W = img.shape
    gx, gy = _grad_mag(img)
    if score == "grad":
        sc = gx * gx + gy * gy
    else:
        ixx = _box3(gx * gx)
        iyy = _box3(gy * gy)
        ixy = _box3(gx * gy)
        sc = ixx * iyy - ixy * ixy - np.float32(0.04) * (ixx + iyy) ** 2
    Hv, Wv = H, W
    if ref_shape is not None:
        Hv, Wv = min(H, ref_shape[0]), min(W, ref_shape[1])
    y_lo, y_hi = margin_y, Hv - margin_y
    x_lo, x_hi = margin_x, Wv - margin_x
    pts = []
    if y_hi <= y_lo or x_hi <= x_lo:
        return np.zeros((0, 2), np.int32)
    ys = np.linspace(0, H, grid_y + 1).astype(np.int64)
    xs = np.linspace(0, W, grid_x + 1).astype(np.int64)
    for gyi in range(grid_y):
        a0, a1 = max(ys[gyi], y_lo), min(ys[gyi + 1], y_hi)
        if a1 <= a0:
            continue
        for gxi in range(grid_x):
            b0, b1 = max(xs[gxi], x_lo), min(xs[gxi + 1], x_hi)
            if b1 <= b0:
                continue
            cell = sc[a0:a1, b0:b1]
            k = int(np.argmax(cell))
            py, px = divmod(k, cell.shape[1])
            pts.append((b0 + px, a0 + py))
    return np.asarray(pts, np.int32).reshape(-1, 2)


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------


@dataclass
class Pair:
    ref: np.ndarray            # float32 [H][W] in [0, 1]
    sen: np.ndarray            # float32 [Hs][Ws] in [0, 1]
    points: np.ndarray         # int32 (n, 2) (x, y) in sensed coordinates
    m: int                     # template side
    R: int                     # search radius
    truth: np.ndarray          # float64 (n, 2): true (dx, dy) of each point
    meta: dict = field(default_factory=dict)


def template_half(m):
    """Rows/cols before the centre: (m-1)//2 for odd m, m//2 for even m."""
    return (m - 1) // 2 if m % 2 == 1 else m // 2


def margin_for(m, R):
    h = template_half(m)
    return h + R, (m - 1 - h) + R


def _points_for(sen, ref_shape, m, R, grid, score, n_max=None):
    lo, hi = margin_for(m, R)
    mg = max(lo, hi) + 1
    pts = block_points(sen, grid[0], grid[1], mg, mg, score=score, ref_shape=ref_shape)
    if n_max is not None:
        pts = pts[:n_max]
    return pts


def inverting_pair_512(seed=1000, H=512, W=512, n_side=10, m=41, R=10, max_shift=8):
    """512^2 reference from value noise + 30 rectangles + 20 lines; sensed is
    a monotone-then-inverting piecewise map of the reference shifted by an
    integer (sx, sy) in [-8, 8]^2; 100 block-max points; m=41, R=10."""
    rng = np.random.default_rng(seed)
    ref = optical_like(rng, H, W, n_rects=30, n_lines=20)
    sx, sy = (int(v) for v in rng.integers(-max_shift, max_shift + 1, 2))
    f, knot = piecewise_inverting_map(rng)
    sen = scale01(f(shift_image(ref, sx, sy)))
    pts = _points_for(sen, ref.shape, m, R, (n_side, n_side), "grad")
    truth = np.tile(np.array([[-sx, -sy]], np.float64), (len(pts), 1))
    return Pair(ref, sen, pts, m, R, truth, dict(shift=(sx, sy), knot=knot, seed=seed))


def sar_pair_2048(seed=2000, H=2048, W=2048, grid=32, n_points=1000, m=81, R=20,
            max_shift=15, block=256, looks=4):
    """2048^2 optical-like reference; SAR-like sensed image: nonlinear remap,
    Gamma speckle with L=4 looks, and a piecewise-constant shift field with
    256-px blocks and integer offsets in [-15, 15]^2; 1000 block-Harris
    points on a 32x32 grid; m=81, R=20."""
    rng = np.random.default_rng(seed)
    ref = optical_like(rng, H, W)
    nby = -(-H // block)
    nbx = -(-W // block)
    offs = rng.integers(-max_shift, max_shift + 1, size=(nby, nbx, 2))
    g = float(rng.uniform(0.5, 2.0))
    remapped = np.power(ref, np.float32(g)) * np.float32(0.8) + np.float32(0.2) * np.sin(
        np.float32(3.0 * math.pi) * ref).astype(np.float32) ** 2
    shifted = shift_field_image(remapped.astype(np.float32), block, offs)
    sen = scale01(shifted * gamma_speckle(rng, shifted.shape, looks))
    pts = _points_for(sen, ref.shape, m, R, (grid, grid), "harris", n_points)
    bidx = np.stack([pts[:, 1] // block, pts[:, 0] // block], 1) if len(pts) else np.zeros((0, 2), int)
    truth = -offs[bidx[:, 0], bidx[:, 1]].astype(np.float64) if len(pts) else np.zeros((0, 2))
    return Pair(ref, sen, pts, m, R, truth, dict(gamma=g, block=block, seed=seed))


def _mixed_pair(seed, p, side_lo, side_hi, templates, r_lo, r_hi, pts_lo, pts_hi, max_shift, scale):
    """Pair p of the mixed batch, drawn from its own seed (seed + 1 + p) only."""
    kinds = ("linear", "gamma", "inverted", "speckled")
    prng = np.random.default_rng(seed + 1 + p)
    H = int(prng.integers(side_lo, side_hi + 1) * scale)
    W = int(prng.integers(side_lo, side_hi + 1) * scale)
    m = int(templates[int(prng.integers(0, len(templates)))])
    R = int(prng.integers(r_lo, r_hi + 1))
    npts = int(prng.integers(pts_lo, pts_hi + 1) * scale)
    kind = kinds[int(prng.integers(0, 4))]
    H = max(H, m + 2 * R + 8)
    W = max(W, m + 2 * R + 8)
    ref = optical_like(prng, H, W)
    sx, sy = (int(v) for v in prng.integers(-max_shift, max_shift + 1, 2))
    sen = radiometric(prng, shift_image(ref, sx, sy), kind)
    g = max(1, int(math.ceil(math.sqrt(max(1, npts)))))
    pts = _points_for(sen, ref.shape, m, R, (g, g), "grad", npts)
    truth = np.tile(np.array([[-sx, -sy]], np.float64), (len(pts), 1))
    return Pair(ref, sen, pts, m, R, truth, dict(kind=kind, shift=(sx, sy), seed=seed + 1 + p))


def mixed_batch(seed=4000, n_pairs=64, side_lo=512, side_hi=4096, templates=(41, 61, 81, 101),
                r_lo=10, r_hi=40, pts_lo=200, pts_hi=4000, max_shift=8, scale=1.0, workers=1):
    """64 pairs, sides uniform in [512, 4096] (non-square allowed), each with
    one radiometric map of {linear, gamma, inverted, speckled}, 200-4000
    points, m from {41, 61, 81, 101}, R uniform in [10, 40].  ``scale``
    shrinks sides and point counts for quick variants (1.0 = the full size).
    Each pair depends on its own seed only, so ``workers`` > 1 builds them in
    parallel processes (started with ``spawn``) with the same result."""
    args = [(seed, p, side_lo, side_hi, templates, r_lo, r_hi, pts_lo, pts_hi, max_shift, scale)
            for p in range(n_pairs)]
    if workers <= 1 or n_pairs <= 1:
        return [_mixed_pair(*a) for a in args]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=min(workers, n_pairs), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_mixed_pair, *zip(*args)))


def speckle_pair_10000(seed=5000, H=10000, W=10000, n_points=10000, m=101, R=40, block=512,
            max_rot_deg=1.0, scale_lo=0.99, scale_hi=1.01, max_translation=28, looks=1):
    """10000^2 uint16 reference (converted to float32 / 65535); the sensed
    image is an L=1 Gamma-speckled, bilinearly resampled copy under a
    per-block affine residual (rotation <= 1 deg, scale 0.99-1.01 about each
    512-px block centre) plus a per-block translation, keeping the total
    displacement within 40 px; 10000 points; m=101, R=40."""
    rng = np.random.default_rng(seed)
    ref16 = np.round(optical_like(rng, H, W) * np.float32(65535.0)).astype(np.uint16)
    ref = (ref16.astype(np.float32) / np.float32(65535.0)).astype(np.float32)
    nby = -(-H // block)
    nbx = -(-W // block)
    rot = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, (nby, nbx)))
    scl = rng.uniform(scale_lo, scale_hi, (nby, nbx))
    trn = rng.integers(-max_translation, max_translation + 1, (nby, nbx, 2))
    sen = np.empty_like(ref)
    for by in range(nby):
        y0, y1 = by * block, min(H, (by + 1) * block)
        yy = np.arange(y0, y1, dtype=np.float64)[:, None]
        for bx in range(nbx):
            x0, x1 = bx * block, min(W, (bx + 1) * block)
            xx = np.arange(x0, x1, dtype=np.float64)[None, :]
            cy, cx = (y0 + y1) / 2.0, (x0 + x1) / 2.0
            c, s = math.cos(rot[by, bx]) * scl[by, bx], math.sin(rot[by, bx]) * scl[by, bx]
            dxs = xx - cx
            dys = yy - cy
            src_x = cx + c * dxs - s * dys - trn[by, bx, 0]
            src_y = cy + s * dxs + c * dys - trn[by, bx, 1]
            sen[y0:y1, x0:x1] = bilinear_sample(ref, src_y, src_x)
    sen = scale01(sen * gamma_speckle(rng, sen.shape, looks))
    g = int(math.ceil(math.sqrt(n_points)))
    pts = _points_for(sen, ref.shape, m, R, (g, g), "grad", n_points)
    # true displacement d(p) = source(p) - p for each point
    truth = np.zeros((len(pts), 2), np.float64)
    for k, (px, py) in enumerate(pts):
        by, bx = py // block, px // block
        y0, x0 = by * block, bx * block
        y1, x1 = min(H, y0 + block), min(W, x0 + block)
        cy, cx = (y0 + y1) / 2.0, (x0 + x1) / 2.0
        c, s = math.cos(rot[by, bx]) * scl[by, bx], math.sin(rot[by, bx]) * scl[by, bx]
        sxp = cx + c * (px - cx) - s * (py - cy) - trn[by, bx, 0]
        syp = cy + s * (px - cx) + c * (py - cy) - trn[by, bx, 1]
        truth[k] = (sxp - px, syp - py)
    return Pair(ref, sen, pts, m, R, truth, dict(seed=seed, ref_u16=ref16))


def tiny_pair(seed, H, W, m, R, n_points, shift=(0, 0), kind="piecewise"):
    """Small pair for fast parity cases (ragged sizes, edge cases)."""
    rng = np.random.default_rng(seed)
    ref = optical_like(rng, H, W, n_rects=max(2, H * W // 8000), n_lines=max(2, H * W // 12000))
    sx, sy = shift
    sh = shift_image(ref, sx, sy)
    if kind == "piecewise":
        f, _ = piecewise_inverting_map(rng)
        sen = scale01(f(sh))
    elif kind == "identity":
        sen = sh.copy()
    else:
        sen = radiometric(rng, sh, kind)
    g = max(1, int(math.ceil(math.sqrt(max(1, n_points)))))
    pts = _points_for(sen, ref.shape, m, R, (g, g), "grad", n_points)
    truth = np.tile(np.array([[-sx, -sy]], np.float64), (len(pts), 1))
    return Pair(np.ascontiguousarray(ref), np.ascontiguousarray(sen), pts, m, R, truth, dict(seed=seed))


# ---------------------------------------------------------------------------
# control-point sets for outlier rejection: correspondences under a planted
# model with outliers, and the minimal samples (random draws) of RANSAC
# ---------------------------------------------------------------------------
def planted_model(rng, projective=True):
    """A near-identity planted model (3 x 3, last entry 1): small rotation /
    shear / scale, a translation of up to 40 px and, if projective, a small
    perspective row."""
    H = np.eye(3)
    H[0, 0] += rng.uniform(-0.02, 0.02)
    H[1, 1] += rng.uniform(-0.02, 0.02)
    H[0, 1] = rng.uniform(-0.02, 0.02)
    H[1, 0] = rng.uniform(-0.02, 0.02)
    H[0, 2] = rng.uniform(-40, 40)
    H[1, 2] = rng.uniform(-40, 40)
    if projective:
        H[2, 0] = rng.uniform(-2e-5, 2e-5)
        H[2, 1] = rng.uniform(-2e-5, 2e-5)
    return H


def apply_model(H, pts):
    q = np.c_[pts, np.ones(len(pts))] @ np.asarray(H).T
    return q[:, :2] / q[:, 2:]


def planted_correspondences(seed, n, projective=True, outlier_frac=0.3, noise=0.0, extent=2000.0):
    """n source points uniform in [0, extent)^2; destinations = the planted
    model applied to them (plus Gaussian noise of std `noise` px); a fraction
    replaced by outliers 20-200 px off their planted position.  Returns
    (src, dst, H0, is_outlier)."""
    rng = np.random.default_rng(seed)
    H0 = planted_model(rng, projective)
    src = rng.uniform(0, extent, (n, 2))
    dst = apply_model(H0, src)
    if noise > 0:
        dst = dst + rng.normal(0, noise, dst.shape)
    out = rng.random(n) < outlier_frac
    k = int(out.sum())
    dst[out] += rng.uniform(20, 200, (k, 2)) * rng.choice([-1.0, 1.0], (k, 2))
    return src, dst, H0, out


def ransac_samples(seed, n, n_hyp, k):
    """n_hyp minimal samples of k distinct indices in [0, n): the random
    draws of RANSAC, passed to both the oracle and the kernels."""
    rng = np.random.default_rng(seed)
    s = np.empty((n_hyp, k), np.int32)
    for h in range(n_hyp):
        s[h] = rng.choice(n, k, replace=False)
    return s
