"""FP64 CPU oracle for SFOC + Fast-NCC_SFOC (arXiv 2202.13347, Sec. 2).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` and by
nothing else; the product library under ``paper_2202_13347_gb300/`` never
imports it and shares no code with it.

The arithmetic lives in ``sfoc_oracle.c`` (plain loops, double precision,
OpenMP over independent pixels/points).  This module only compiles it
(``build()``) and marshals numpy arrays through ctypes.

Function map (paper citation in each C function's comment):
  sfoc_roi     Eq. 1-7 + dilated smoothing and normalisation (Sec. 2.1)
  match        Eq. 8 evaluated literally, argmax, parabola sub-pixel
  ncc_eq9_dft  Eq. 9 with Eq. 13 (naive DFT) and Eq. 14-16 (tiny inputs)
  integral     Eq. 14-15 (exclusive prefix), rect_sum Eq. 16
  kernel_*     Eq. 2, 3, 5 and the dilated Gaussian
  ransac       RANSAC with a projective / affine model (Sec. 3.2.3)
  match_quality  NCM, CMR and the RMSE of Eq. 22 (Sec. 4.1)
  fast_score / fast_blocks  block-based FAST interest points (Sec. 3.1.1)
  rectify      bilinear resampling of the sensed image with the model (Sec. 3.2.3)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfoc_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "ransac_oracle.c"), os.path.join(_HERE, "fast_oracle.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
# A prebuilt oracle library to load instead of the in-tree build: the
# mutation tests point this at builds with one planted mistake each.
_LIB_OVERRIDE = os.environ.get("SFOC_ORACLE_LIB")

# status codes (values fixed by the paper-derived conventions, independent of
# the CUDA library's header)
OK, OUT_OF_BOUNDS, FLAT_TEMPLATE, PEAK_ON_EDGE, NAN_INPUT = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 -fopenmp (plain C, portable)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("n_scales", C.c_int),
        ("scales", C.c_double * 8),
        ("sigma2", C.c_double),
        ("n_orient", C.c_int),
        ("n_dil", C.c_int),
        ("dil", C.c_int * 4),
        ("sigma_d1", C.c_double),
        ("sigma_d2", C.c_double),
        ("eps", C.c_double),
        ("rectify", C.c_int),
        ("radius_mult", C.c_double),
        ("first_order_only", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [
        ("dx", C.c_int32), ("dy", C.c_int32), ("ncc", C.c_double),
        ("sub_dx", C.c_double), ("sub_dy", C.c_double), ("status", C.c_int32),
        ("margin", C.c_double),
    ]


class Cube(C.Structure):
    _fields_ = [
        ("data", C.POINTER(C.c_double)),
        ("z", C.c_int), ("H", C.c_int), ("W", C.c_int),
        ("roi_y0", C.c_int), ("roi_x0", C.c_int), ("roi_h", C.c_int), ("roi_w", C.c_int),
    ]


def params(scales=(0.6, 0.8, 1.0), sigma2=1.5, n_orient=6, dil=(1, 2, 3), sigma_d1=1.0,
           sigma_d2=1.5, eps=1e-3, rectify=True, radius_mult=3.0, first_order_only=False) -> Params:
    """Paper defaults: Table 2 STDs, 6 orientations and rates {1,2,3} (Sec. 2.1).
    Variants: first_order_only (F-SFOC, Sec. 4.2); dil=(1,) (a plain
    Gaussian, Fig. 3 (e)); sigma_d1 / sigma_d2 = 0 (that group unsmoothed,
    Fig. 3 (d))."""
    p = Params()
    p.n_scales = len(scales)
    for i, s in enumerate(scales):
        p.scales[i] = float(s)
    p.sigma2 = float(sigma2)
    p.n_orient = int(n_orient)
    p.n_dil = len(dil)
    for i, r in enumerate(dil):
        p.dil[i] = int(r)
    p.sigma_d1 = float(sigma_d1)
    p.sigma_d2 = float(sigma_d2)
    p.eps = float(eps)
    p.rectify = 1 if rectify else 0
    p.radius_mult = float(radius_mult)
    p.first_order_only = 1 if first_order_only else 0
    return p


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.oracle_radius.restype = C.c_int
        L.oracle_radius.argtypes = [C.c_double, C.c_double]
        L.oracle_channels.restype = C.c_int
        L.oracle_channels.argtypes = [C.POINTER(Params)]
        L.oracle_num_threads.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_kernel_g1.argtypes = [C.c_double, C.c_int, dp, dp]
        L.oracle_kernel_g2.argtypes = [C.c_double, C.c_int, dp, dp, dp]
        L.oracle_kernel_dilated.argtypes = [C.c_double, C.c_int, C.c_int, dp]
        L.oracle_conv2d.argtypes = [dp, C.c_int, C.c_int, dp, C.c_int, dp]
        L.oracle_sfoc_roi.restype = C.c_int
        L.oracle_sfoc_roi.argtypes = [C.POINTER(C.c_float), C.c_int, C.c_int, C.POINTER(Params),
                                      C.c_int, C.c_int, C.c_int, C.c_int, dp]
        L.oracle_integral.argtypes = [dp, C.c_int, C.c_int, dp]
        L.oracle_rect_sum.restype = C.c_double
        L.oracle_rect_sum.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.oracle_template_half.restype = C.c_int
        L.oracle_template_half.argtypes = [C.c_int]
        L.oracle_parabola.restype = C.c_double
        L.oracle_parabola.argtypes = [C.c_double, C.c_double, C.c_double]
        L.oracle_pick.argtypes = [dp, C.c_int, C.POINTER(Result)]
        L.oracle_match.restype = C.c_int
        L.oracle_match.argtypes = [C.POINTER(Cube), C.POINTER(Cube), C.POINTER(C.c_int32), C.c_int,
                                   C.c_int, C.c_int, C.POINTER(Result), dp]
        L.oracle_complexity_ratio.restype = C.c_double
        L.oracle_complexity_ratio.argtypes = [C.c_int] * 5
        L.oracle_ncc_eq9_dft.restype = C.c_int
        L.oracle_ncc_eq9_dft.argtypes = [dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, dp]
        up = C.POINTER(C.c_uint8)
        ip = C.POINTER(C.c_int)
        L.oracle_ransac.restype = C.c_int
        L.oracle_ransac.argtypes = [dp, dp, up, C.c_int, C.c_int, ip, C.c_int, C.c_double, C.c_int, dp, up, ip, ip,
                                    ip]
        L.oracle_ransac_fit.restype = C.c_int
        L.oracle_ransac_fit.argtypes = [dp, dp, up, C.c_int, C.c_int, ip, dp]
        L.oracle_match_quality.restype = C.c_int
        L.oracle_match_quality.argtypes = [dp, dp, dp, up, C.c_int, C.c_double, dp, dp]
        fp = C.POINTER(C.c_float)
        L.oracle_rectify.restype = C.c_int
        L.oracle_rectify.argtypes = [fp, C.c_int, C.c_int, dp, C.c_float, C.c_int, C.c_int, fp]
        L.oracle_fast_score.argtypes = [fp, C.c_int, C.c_int, C.c_float, fp]
        L.oracle_fast_blocks.restype = C.c_int
        L.oracle_fast_blocks.argtypes = [fp, C.c_int, C.c_int, C.c_float, C.c_int, C.c_int, C.c_int,
                                         C.POINTER(C.c_int32), fp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def radius(sigma, mult=3.0) -> int:
    return lib().oracle_radius(float(sigma), float(mult))


def channels(p: Params) -> int:
    return lib().oracle_channels(C.byref(p))


def kernel_g1(sigma, K):
    n = 2 * K + 1
    gx = np.zeros((n, n)); gy = np.zeros((n, n))
    lib().oracle_kernel_g1(float(sigma), int(K), _dp(gx), _dp(gy))
    return gx, gy


def kernel_g2(sigma, K):
    n = 2 * K + 1
    a = np.zeros((n, n)); b = np.zeros((n, n)); c = np.zeros((n, n))
    lib().oracle_kernel_g2(float(sigma), int(K), _dp(a), _dp(b), _dp(c))
    return a, b, c


def kernel_dilated(sigma_d, Kd, r):
    n = 2 * r * Kd + 1
    w = np.zeros((n, n))
    lib().oracle_kernel_dilated(float(sigma_d), int(Kd), int(r), _dp(w))
    return w


def conv2d(img, k):
    img = np.ascontiguousarray(img, np.float64)
    k = np.ascontiguousarray(k, np.float64)
    K = (k.shape[0] - 1) // 2
    out = np.zeros_like(img)
    lib().oracle_conv2d(_dp(img), img.shape[0], img.shape[1], _dp(k), K, _dp(out))
    return out


@dataclass
class CubeROI:
    data: np.ndarray   # float64 [z][h][w]
    H: int
    W: int
    y0: int
    x0: int

    def cstruct(self) -> Cube:
        c = Cube()
        c.data = _dp(self.data)
        c.z, c.H, c.W = self.data.shape[0], self.H, self.W
        c.roi_y0, c.roi_x0 = self.y0, self.x0
        c.roi_h, c.roi_w = self.data.shape[1], self.data.shape[2]
        return c


def sfoc_roi(image, p: Params = None, y0=0, x0=0, h=None, w=None) -> CubeROI:
    """SFOC cube of ``image`` on [y0, y0+h) x [x0, x0+w) (default: whole)."""
    if p is None:
        p = params()
    img = np.ascontiguousarray(image, np.float32)
    H, W = img.shape
    h = H - y0 if h is None else h
    w = W - x0 if w is None else w
    z = channels(p)
    out = np.zeros((z, h, w), np.float64)
    rc = lib().oracle_sfoc_roi(img.ctypes.data_as(C.POINTER(C.c_float)), H, W, C.byref(p),
                               int(y0), int(x0), int(h), int(w), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle_sfoc_roi failed: %d" % rc)
    return CubeROI(out, H, W, int(y0), int(x0))


def sfoc(image, p: Params = None) -> np.ndarray:
    return sfoc_roi(image, p).data


def template_half(m: int) -> int:
    return lib().oracle_template_half(int(m))


def match(ref: CubeROI, sen: CubeROI, points, m: int, R: int, want_maps=False):
    """Eq. 8 matching.  Returns a structured dict of numpy arrays (and the
    (n, 2R+1, 2R+1) NCC maps when ``want_maps``)."""
    pts = np.ascontiguousarray(points, np.int32).reshape(-1, 2)
    n = pts.shape[0]
    res = (Result * max(1, n))()
    P1 = 2 * R + 1
    maps = np.zeros((max(1, n), P1, P1), np.float64) if want_maps else None
    rc_ = ref.cstruct(); sc_ = sen.cstruct()
    rc = lib().oracle_match(C.byref(rc_), C.byref(sc_), pts.ctypes.data_as(C.POINTER(C.c_int32)), n,
                            int(m), int(R), res, _dp(maps) if want_maps else None)
    if rc != 0:
        raise RuntimeError("oracle_match failed: %d" % rc)
    out = dict(
        dx=np.array([res[i].dx for i in range(n)], np.int32),
        dy=np.array([res[i].dy for i in range(n)], np.int32),
        ncc=np.array([res[i].ncc for i in range(n)], np.float64),
        sub_dx=np.array([res[i].sub_dx for i in range(n)], np.float64),
        sub_dy=np.array([res[i].sub_dy for i in range(n)], np.float64),
        status=np.array([res[i].status for i in range(n)], np.int32),
        margin=np.array([res[i].margin for i in range(n)], np.float64),
    )
    if want_maps:
        out["maps"] = maps[:n]
    return out


def pick(ncc_map):
    m = np.ascontiguousarray(ncc_map, np.float64)
    R = (m.shape[0] - 1) // 2
    r = Result()
    lib().oracle_pick(_dp(m), R, C.byref(r))
    return dict(dx=r.dx, dy=r.dy, ncc=r.ncc, sub_dx=r.sub_dx, sub_dy=r.sub_dy, status=r.status, margin=r.margin)


def parabola(cm, c0, cp) -> float:
    return lib().oracle_parabola(float(cm), float(c0), float(cp))


def complexity_ratio(z, m, n, M, N) -> float:
    """Eq. 19: T1/T2 with T1 from Eq. 17 and T2 from Eq. 18."""
    return lib().oracle_complexity_ratio(int(z), int(m), int(n), int(M), int(N))


def integral(g):
    g = np.ascontiguousarray(g, np.float64)
    H, W = g.shape
    P = np.zeros((H + 1, W + 1))
    lib().oracle_integral(_dp(g), H, W, _dp(P))
    return P


def rect_sum(P, y0, x0, y1, x1) -> float:
    P = np.ascontiguousarray(P, np.float64)
    return lib().oracle_rect_sum(_dp(P), P.shape[1] - 1, int(y0), int(x0), int(y1), int(x1))


def ncc_eq9_dft(S, T, R, L=None):
    S = np.ascontiguousarray(S, np.float64)
    T = np.ascontiguousarray(T, np.float64)
    z, m = T.shape[0], T.shape[1]
    M = m + 2 * R
    if L is None:
        L = M
    P1 = 2 * R + 1
    out = np.zeros((P1, P1))
    rc = lib().oracle_ncc_eq9_dft(_dp(S), _dp(T), z, m, R, int(L), _dp(out))
    if rc != 0:
        raise RuntimeError("oracle_ncc_eq9_dft failed: %d" % rc)
    return out


def match_pair(ref_img, sen_img, points, m, R, p: Params = None, want_maps=False, roi=True):
    """SFOC of both images (only on the rectangles the windows need when
    ``roi``) followed by Eq. 8 matching, one point at a time."""
    if p is None:
        p = params()
    pts = np.ascontiguousarray(points, np.int32).reshape(-1, 2)
    if not roi:
        rc = sfoc_roi(ref_img, p)
        sc = sfoc_roi(sen_img, p)
        return match(rc, sc, pts, m, R, want_maps)
    h = template_half(m)
    Hr, Wr = ref_img.shape
    Hs, Ws = sen_img.shape
    outs = []
    for k in range(pts.shape[0]):
        px, py = int(pts[k, 0]), int(pts[k, 1])
        ty0, tx0 = py - h, px - h
        ok = (ty0 >= 0 and tx0 >= 0 and ty0 + m <= Hs and tx0 + m <= Ws and ty0 - R >= 0 and tx0 - R >= 0
              and ty0 + m + R <= Hr and tx0 + m + R <= Wr)
        if not ok:
            rc_roi = CubeROI(np.zeros((channels(p), 1, 1)), Hr, Wr, 0, 0)
            sc_roi = CubeROI(np.zeros((channels(p), 1, 1)), Hs, Ws, 0, 0)
        else:
            rc_roi = sfoc_roi(ref_img, p, ty0 - R, tx0 - R, m + 2 * R, m + 2 * R)
            sc_roi = sfoc_roi(sen_img, p, ty0, tx0, m, m)
        outs.append(match(rc_roi, sc_roi, pts[k:k + 1], m, R, want_maps))
    keys = ["dx", "dy", "ncc", "sub_dx", "sub_dy", "status", "margin"] + (["maps"] if want_maps else [])
    if not outs:
        return {k: np.zeros((0,)) for k in keys}
    return {k: np.concatenate([o[k] for o in outs]) for k in keys}


# ---------------------------------------------------------------------------
# outlier rejection (Sec. 3.2.3) and matching criteria (Sec. 4.1)
# ---------------------------------------------------------------------------
PROJECTIVE, AFFINE = 1, 0


def _pts(a):
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1, 2))


def _mask(valid, n):
    if valid is None:
        return None, None
    v = np.ascontiguousarray(np.asarray(valid, np.uint8).reshape(n))
    return v, v.ctypes.data_as(C.POINTER(C.c_uint8))


def ransac(src, dst, samples, valid=None, model=PROJECTIVE, tau=1.5, refits=1):
    """RANSAC over correspondences src -> dst (n x 2, pixels) with the given
    minimal samples (n_hyp x 4, or x 3 for the affine model).  Returns
    H (3 x 3), inlier mask, per-hypothesis scores, winning hypothesis and
    inlier count."""
    src, dst = _pts(src), _pts(dst)
    n = len(src)
    k = 4 if model == PROJECTIVE else 3
    samp = np.ascontiguousarray(np.asarray(samples, np.int32).reshape(-1, k))
    v, vp = _mask(valid, n)
    H = np.zeros(9)
    inl = np.zeros(n, np.uint8)
    scores = np.zeros(len(samp), np.int32)
    best, cnt = C.c_int(0), C.c_int(0)
    ip = C.POINTER(C.c_int)
    rc = lib().oracle_ransac(_dp(src), _dp(dst), vp, n, int(model), samp.ctypes.data_as(ip), len(samp), float(tau),
                             int(refits), _dp(H), inl.ctypes.data_as(C.POINTER(C.c_uint8)),
                             scores.ctypes.data_as(ip), C.byref(best), C.byref(cnt))
    if rc != 0:
        raise ValueError("oracle_ransac: bad arguments")
    return dict(H=H.reshape(3, 3), inlier=inl.astype(bool), scores=scores, best=best.value, count=cnt.value)


def ransac_fit(src, dst, idx, valid=None, model=PROJECTIVE):
    """The exact model on one minimal sample (None when singular)."""
    src, dst = _pts(src), _pts(dst)
    v, vp = _mask(valid, len(src))
    ix = np.ascontiguousarray(np.asarray(idx, np.int32))
    H = np.zeros(9)
    ok = lib().oracle_ransac_fit(_dp(src), _dp(dst), vp, len(src), int(model),
                                 ix.ctypes.data_as(C.POINTER(C.c_int)), _dp(H))
    return H.reshape(3, 3) if ok else None


def match_quality(P, src, dst, valid=None, tau=1.5):
    """NCM, CMR and RMSE (Eq. 22) of the matches src -> dst against model P."""
    src, dst = _pts(src), _pts(dst)
    v, vp = _mask(valid, len(src))
    Pm = np.ascontiguousarray(np.asarray(P, np.float64).reshape(9))
    cmr, rmse = C.c_double(0), C.c_double(0)
    ncm = lib().oracle_match_quality(_dp(Pm), _dp(src), _dp(dst), vp, len(src), float(tau), C.byref(cmr),
                                     C.byref(rmse))
    return dict(ncm=ncm, cmr=cmr.value, rmse=rmse.value)


# ---------------------------------------------------------------------------
# block-based FAST interest points (Sec. 3.1.1)
# ---------------------------------------------------------------------------
def _img32(img):
    return np.ascontiguousarray(np.asarray(img, np.float32))


def fast_score(img, t=0.05):
    """FAST-9 score of every pixel (0 where it is no corner)."""
    a = _img32(img)
    H, W = a.shape
    out = np.zeros((H, W), np.float32)
    fp = C.POINTER(C.c_float)
    lib().oracle_fast_score(a.ctypes.data_as(fp), H, W, C.c_float(t), out.ctypes.data_as(fp))
    return out


def fast_blocks(img, t=0.05, grid_y=8, grid_x=8, margin=3):
    """One FAST point per block: points (grid_y * grid_x, 2) int32 (x, y;
    -1 where a block has none), scores (grid_y * grid_x,) float32."""
    a = _img32(img)
    H, W = a.shape
    nb = grid_y * grid_x
    pts = np.zeros((nb, 2), np.int32)
    sc = np.zeros(nb, np.float32)
    fp = C.POINTER(C.c_float)
    rc = lib().oracle_fast_blocks(a.ctypes.data_as(fp), H, W, C.c_float(t), int(grid_y), int(grid_x), int(margin),
                                  pts.ctypes.data_as(C.POINTER(C.c_int32)), sc.ctypes.data_as(fp))
    if rc < 0:
        raise ValueError("oracle_fast_blocks: bad arguments")
    return pts, sc


def rectify(img, H, out_shape=None, fill=0.0):
    """The sensed image resampled into the reference frame with the model H
    (sensed -> reference), bilinear; out_shape defaults to img.shape."""
    a = np.ascontiguousarray(np.asarray(img, np.float32))
    h, w = a.shape
    oh, ow = out_shape or (h, w)
    Hm = np.ascontiguousarray(np.asarray(H, np.float64).reshape(9))
    out = np.zeros((oh, ow), np.float32)
    fp = C.POINTER(C.c_float)
    rc = lib().oracle_rectify(a.ctypes.data_as(fp), h, w, _dp(Hm), C.c_float(fill), oh, ow, out.ctypes.data_as(fp))
    if rc != 0:
        raise ValueError("singular model")
    return out
