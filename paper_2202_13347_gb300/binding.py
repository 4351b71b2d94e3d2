"""Thin ctypes binding of libsfoc_gb300.so (include/sfoc.h).

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  Torch supplies device memory (tensor data pointers) and the
stream.  If the library is missing the import of this module fails loudly;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfoc_gb300.so")

OK = 0
ERR_NAMES = {0: "SFOC_OK", -1: "SFOC_ERR_INVALID_ARG", -2: "SFOC_ERR_SHAPE", -3: "SFOC_ERR_OOM",
             -4: "SFOC_ERR_CUDA", -5: "SFOC_ERR_TIMEOUT", -6: "SFOC_ERR_UNSUPPORTED"}
PT_OK, PT_OUT_OF_BOUNDS, PT_FLAT_TEMPLATE, PT_PEAK_ON_EDGE, PT_NAN = 0, 1, 2, 3, 4
DTYPE_F32, DTYPE_BF16 = 0, 1
(CORR_AUTO, CORR_DIRECT_F32, CORR_IGEMM_TC, CORR_TC_TOEPLITZ, CORR_TC_COLUMN, CORR_TC_BAND,
 CORR_FFT) = 0, 1, 2, 3, 4, 5, 6
MODEL_AFFINE, MODEL_PROJECTIVE = 0, 1
STATIC_SCRATCH_FLOATS = 1 << 24  # SFOC_STATIC_SCRATCH_FLOATS


class SfocError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


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
        ("cube_dtype", C.c_int),
    ]


class Result(C.Structure):
    _fields_ = [("dx", C.c_int32), ("dy", C.c_int32), ("ncc", C.c_float), ("sub_dx", C.c_float),
                ("sub_dy", C.c_float), ("status", C.c_int32)]


class Peaks(C.Structure):
    _fields_ = [("fp32_tflops", C.c_double), ("fp32x2_tflops", C.c_double), ("fp64_tflops", C.c_double),
                ("hbm_copy_gbs", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("corr_path", C.c_int), ("d_maps", C.c_void_p)]


_lib = None

# every function of include/sfoc.h with (restype, argtypes)
_P = C.c_void_p
_SIGS = {
    "sfoc_ctx_create": (C.c_int, [C.POINTER(_P), C.c_int, _P]),
    "sfoc_ctx_destroy": (C.c_int, [_P]),
    "sfoc_ctx_set_stream": (C.c_int, [_P, _P]),
    "sfoc_ctx_sync": (C.c_int, [_P]),
    "sfoc_ctx_selftest_timeout": (C.c_int, [_P, C.c_int]),
    "sfoc_ctx_reserve": (C.c_int, [_P, C.c_size_t]),
    "sfoc_match_workspace_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "sfoc_last_error_string": (C.c_char_p, [_P]),
    "sfoc_ctx_launch_count": (C.c_int64, [_P]),
    "sfoc_ctx_enable_timing": (C.c_int, [_P, C.c_int]),
    "sfoc_ctx_stage_times": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "sfoc_ctx_reset_timing": (C.c_int, [_P]),
    "sfoc_params_default": (C.c_int, [C.POINTER(Params)]),
    "sfoc_measure_peaks": (C.c_int, [_P, C.POINTER(Peaks)]),
    "sfoc_build": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, C.POINTER(C.c_double), C.c_int, C.c_int,
                             C.POINTER(Params), C.POINTER(_P)]),
    "sfoc_cube_info": (C.c_int, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
    "sfoc_cube_export": (C.c_int, [_P, _P, _P]),
    "sfoc_cube_export_integral": (C.c_int, [_P, _P, _P]),
    "sfoc_cube_free": (C.c_int, [_P]),
    "fastncc_match": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, C.c_int, C.POINTER(Opts), _P]),
    "fastncc_register_pair": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, C.c_int, C.c_int, _P, C.c_int, C.c_int,
                                        C.c_int, C.POINTER(Params), C.POINTER(Opts), _P]),
    "fastncc_register_pair_host": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, C.c_int, C.c_int, _P, C.c_int,
                                             C.c_int, C.c_int, C.POINTER(Params), C.POINTER(Opts), _P]),
    "sfoc_build_u16": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, _P, C.POINTER(_P)]),
    "sfoc_cube_view": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "sfoc_build_static": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, _P, _P]),
    "sfoc_build_batch": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                   C.POINTER(C.c_size_t), C.POINTER(Params), C.POINTER(_P)]),
    "fastncc_match_batch": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                      C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(Opts), C.POINTER(_P)]),
    "fastncc_register_batch": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_P),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.POINTER(Params), C.POINTER(Opts), C.POINTER(_P)]),
    "fastncc_register_batch_host": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                              C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_P),
                                              C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                              C.POINTER(Params), C.POINTER(Opts), C.POINTER(_P)]),
    "fastncc_submit_batch_host": (C.c_int, [_P, C.c_int, C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(_P), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_P),
                                            C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                            C.POINTER(Params), C.POINTER(Opts), C.POINTER(_P),
                                            C.POINTER(C.c_int64)]),
    "fastncc_wait_batch_host": (C.c_int, [_P, C.c_int64]),
    "sfoc_ctx_plan_count": (C.c_int, [_P]),
    "sfoc_ctx_plan_info": (C.c_int, [_P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "sfoc_ctx_stage_scopes": (C.c_int, [_P, C.c_int, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]),
    "sfoc_ctx_release_plans": (C.c_int, [_P]),
    "sfoc_ctx_set_autotune": (C.c_int, [_P, C.c_int]),
    "sfoc_ctx_autotune_entry": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_float), C.POINTER(C.c_int)]),
    "sfoc_ctx_autotune_export": (C.c_int, [_P, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "sfoc_ctx_autotune_import": (C.c_int, [_P, C.c_char_p]),
    "fastncc_points_from_results": (C.c_int, [_P, _P, _P, C.c_int, _P, _P, _P]),
    "sfoc_rectify": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, _P, C.c_float, C.c_int, C.c_int, _P]),
    "sfoc_fast_blocks": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_size_t, C.c_float, C.c_int, C.c_int, C.c_int, _P,
                                   _P]),
    "fastncc_ransac": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_int, _P, C.c_int, C.c_double, C.c_int, _P, _P, _P,
                                 _P]),
}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libsfoc_gb300.so is not built (run paper_2202_13347_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def params(scales=(0.6, 0.8, 1.0), sigma2=1.5, n_orient=6, dil=(1, 2, 3), sigma_d1=1.0, sigma_d2=1.5,
           eps=1e-3, rectify=True, radius_mult=3.0, first_order_only=False, dtype=DTYPE_F32) -> Params:
    """Descriptor parameters; the defaults are the paper's (Sec. 2.1, Table 2).
    Variants: first_order_only (F-SFOC, Sec. 4.2); dil=(1,) (a plain
    Gaussian, Fig. 3 (e)); sigma_d1 / sigma_d2 = 0 (that group unsmoothed,
    Fig. 3 (d))."""
    p = Params()
    lib().sfoc_params_default(C.byref(p))
    p.n_scales = len(scales)
    for i, s in enumerate(scales):
        p.scales[i] = float(s)
    p.sigma2 = float(sigma2)
    p.n_orient = int(n_orient)
    p.n_dil = len(dil)
    for i, r in enumerate(dil):
        p.dil[i] = int(r)
    p.sigma_d1, p.sigma_d2, p.eps = float(sigma_d1), float(sigma_d2), float(eps)
    p.rectify = 1 if rectify else 0
    p.radius_mult = float(radius_mult)
    p.first_order_only = 1 if first_order_only else 0
    p.cube_dtype = int(dtype)
    return p


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _check_shape(t, name, shape):
    """The library reads and writes exactly the elements the sizes it is
    given imply; a tensor of another shape would be read or written past its
    end, so the shape is checked here, before the call."""
    if tuple(t.shape) != tuple(int(v) for v in shape):
        raise ValueError("%s must have shape %s, not %s" % (name, tuple(int(v) for v in shape), tuple(t.shape)))


def _channels(p) -> int:
    """Channels of the cube `p` builds (NULL params = the defaults: 12)."""
    if p is None:
        return 12
    return p.n_orient if p.first_order_only else 2 * p.n_orient


def _check_host(t, name, dtype):
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError("%s must be a contiguous host %s tensor" % (name, dtype))


def _check_cuda(t, name, dtype=None, device=None):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if device is not None and t.device != device:
        # the library runs its kernels on the context's device; a pointer into
        # another GPU's memory is not valid there
        raise ValueError("%s is on %s, the context on %s" % (name, t.device, device))
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s" % (name, dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


class Cube:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle

    def info(self):
        z, H, W, dt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        self.ctx._chk(lib().sfoc_cube_info(self.handle, C.byref(z), C.byref(H), C.byref(W), C.byref(dt)))
        return z.value, H.value, W.value, dt.value

    def export(self) -> torch.Tensor:
        z, H, W, _ = self.info()
        out = torch.empty((z, H, W), dtype=torch.float32, device=self.ctx.device)
        self.ctx._chk(lib().sfoc_cube_export(self.ctx.h, self.handle, _ptr(out)))
        return out

    def view(self):
        """(device address, z, H, W, pitch, dtype) of the cube's own values
        (sfoc_cube_view); the memory stays owned by the cube."""
        d, z, H, W, pitch, dt = C.c_void_p(), C.c_int(), C.c_int(), C.c_int(), C.c_size_t(), C.c_int()
        self.ctx._chk(lib().sfoc_cube_view(self.handle, C.byref(d), C.byref(z), C.byref(H), C.byref(W),
                                           C.byref(pitch), C.byref(dt)))
        return d.value, z.value, H.value, W.value, pitch.value, dt.value

    def export_integral(self) -> torch.Tensor:
        z, H, W, _ = self.info()
        out = torch.empty((2, H + 1, W + 1), dtype=torch.float64, device=self.ctx.device)
        self.ctx._chk(lib().sfoc_cube_export_integral(self.ctx.h, self.handle, _ptr(out)))
        return out

    def free(self):
        if self.handle:
            lib().sfoc_cube_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _results(raw: torch.Tensor):
    return dict(dx=raw[:, 0], dy=raw[:, 1], ncc=raw[:, 2].view(torch.float32),
                sub_dx=raw[:, 3].view(torch.float32), sub_dy=raw[:, 4].view(torch.float32), status=raw[:, 5])


class Context:
    """sfoc_ctx on one device and stream (default: torch's current stream)."""

    def __init__(self, device=0, stream=None):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        idx = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.device = torch.device("cuda", idx)
        if stream is None:
            stream = torch.cuda.current_stream(idx)
        self.stream = stream
        h = C.c_void_p()
        rc = lib().sfoc_ctx_create(C.byref(h), idx, C.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise SfocError(rc, "sfoc_ctx_create failed")
        self.h = h

    def _cuda(self, t, name, dtype=None):
        _check_cuda(t, name, dtype, self.device)

    def _chk(self, rc):
        if rc != OK:
            raise SfocError(rc, lib().sfoc_last_error_string(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().sfoc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        self._chk(lib().sfoc_ctx_set_stream(self.h, C.c_void_p(stream.cuda_stream)))

    def sync(self):
        self._chk(lib().sfoc_ctx_sync(self.h))

    def selftest_timeout(self, limit_us=1000):
        """Enqueues the failure-path self-test (sfoc_ctx_selftest_timeout);
        the next sync() raises SfocError with code -5 (SFOC_ERR_TIMEOUT)."""
        self._chk(lib().sfoc_ctx_selftest_timeout(self.h, int(limit_us)))

    def reserve(self, nbytes):
        self._chk(lib().sfoc_ctx_reserve(self.h, int(nbytes)))

    def measure_peaks(self):
        """This device's FP32 / FP32x2 / FP64 TFLOP/s and HBM copy GB/s,
        measured by the library's microbenchmarks (synchronous)."""
        pk = Peaks()
        self._chk(lib().sfoc_measure_peaks(self.h, C.byref(pk)))
        return {f: getattr(pk, f) for f, _ in Peaks._fields_}

    STAGES = ("steer", "smooth", "integral", "template_stats", "correlation", "ncc_argmax", "other")

    def enable_timing(self, on=True):
        self._chk(lib().sfoc_ctx_enable_timing(self.h, 1 if on else 0))

    def reset_timing(self):
        self._chk(lib().sfoc_ctx_reset_timing(self.h))

    def stage_times(self):
        """{stage: (milliseconds, launches)} accumulated since the last reset."""
        ms = (C.c_double * len(self.STAGES))()
        nl = (C.c_int64 * len(self.STAGES))()
        self._chk(lib().sfoc_ctx_stage_times(self.h, ms, nl))
        return {s: (ms[i], nl[i]) for i, s in enumerate(self.STAGES)}

    @property
    def launch_count(self) -> int:
        return int(lib().sfoc_ctx_launch_count(self.h))

    # -- paper-named calls -------------------------------------------------
    def sfoc_build(self, image: torch.Tensor, scales=None, n_orient=0, p: Params = None, out: Cube = None) -> Cube:
        self._cuda(image, "image", torch.float32)
        H, W = image.shape
        arr = None
        if scales is not None:
            arr = (C.c_double * len(scales))(*[float(s) for s in scales])
        h = C.c_void_p(out.handle if out is not None else None)
        self._chk(lib().sfoc_build(self.h, _ptr(image), H, W, W, arr, len(scales) if scales else 0, int(n_orient),
                                   C.byref(p) if p is not None else None, C.byref(h)))
        if out is not None and h.value == out.handle:
            return out
        return Cube(self, h.value)

    def sfoc_build_u16(self, image: torch.Tensor, p: Params = None, out: Cube = None) -> Cube:
        """sfoc_build of a uint16 image (intensity = value / 65535); torch has
        no uint16 arithmetic, so `image` is passed as an int16 tensor holding
        the same bits."""
        if not (image.is_cuda and image.dtype == torch.int16 and image.is_contiguous()):
            raise ValueError("image must be a contiguous CUDA int16 tensor holding uint16 bits")
        H, W = image.shape
        h = C.c_void_p(out.handle if out is not None else None)
        self._chk(lib().sfoc_build_u16(self.h, _ptr(image), H, W, W, C.byref(p) if p is not None else None,
                                       C.byref(h)))
        if out is not None and h.value == out.handle:
            return out
        return Cube(self, h.value)

    def sfoc_build_static(self, image: torch.Tensor, out: torch.Tensor, p: Params = None) -> torch.Tensor:
        """sfoc_build into the caller's dense float32 [z][H][W] tensor `out`,
        with the library's fixed scratch array instead of the workspace."""
        self._cuda(image, "image", torch.float32)
        self._cuda(out, "out", torch.float32)
        H, W = image.shape
        _check_shape(out, "out", (_channels(p), H, W))
        self._chk(lib().sfoc_build_static(self.h, _ptr(image), H, W, W, C.byref(p) if p is not None else None,
                                          _ptr(out)))
        return out

    def fastncc_match(self, ref: Cube, sen: Cube, points: torch.Tensor, template_size: int, search_radius: int,
                      corr_path=CORR_AUTO, want_maps=False):
        self._cuda(points, "points", torch.int32)
        n = points.shape[0]
        _check_shape(points, "points", (n, 2))
        raw = torch.empty((n, 6), dtype=torch.int32, device=self.device)
        maps = None
        if want_maps:
            P1 = 2 * search_radius + 1
            maps = torch.empty((n, P1, P1), dtype=torch.float32, device=self.device)
        o = Opts(int(corr_path), maps.data_ptr() if maps is not None else None)
        self._chk(lib().fastncc_match(self.h, ref.handle, sen.handle, _ptr(points), n, int(template_size),
                                      int(search_radius), C.byref(o), _ptr(raw)))
        res = _results(raw)
        res["raw"] = raw  # the (n, 6) int32 result rows themselves
        if want_maps:
            res["maps"] = maps
        return res

    def register_pair(self, ref: torch.Tensor, sen: torch.Tensor, points: torch.Tensor, template_size: int,
                      search_radius: int, p: Params = None, corr_path=CORR_AUTO, out: torch.Tensor = None):
        self._cuda(ref, "ref", torch.float32)
        self._cuda(sen, "sen", torch.float32)
        self._cuda(points, "points", torch.int32)
        n = points.shape[0]
        _check_shape(points, "points", (n, 2))
        if out is not None:
            self._cuda(out, "out", torch.int32)
            _check_shape(out, "out", (n, 6))
        raw = out if out is not None else torch.empty((n, 6), dtype=torch.int32, device=self.device)
        o = Opts(int(corr_path), None)
        self._chk(lib().fastncc_register_pair(self.h, _ptr(ref), ref.shape[0], ref.shape[1], _ptr(sen), sen.shape[0],
                                              sen.shape[1], _ptr(points), n, int(template_size), int(search_radius),
                                              C.byref(p) if p is not None else None, C.byref(o), _ptr(raw)))
        return raw

    def register_pair_host(self, ref, sen, points, template_size: int, search_radius: int, p: Params = None,
                           corr_path=CORR_AUTO, out=None):
        """Host (CPU, ideally pinned) tensors in, host results out."""
        _check_host(ref, "ref", torch.float32)
        _check_host(sen, "sen", torch.float32)
        _check_host(points, "points", torch.int32)
        if ref.dim() != 2 or sen.dim() != 2:
            raise ValueError("ref and sen must be 2-D images")
        n = points.shape[0]
        _check_shape(points, "points", (n, 2))
        if out is not None:
            _check_host(out, "out", torch.int32)
            _check_shape(out, "out", (n, 6))
        raw = out if out is not None else torch.empty((n, 6), dtype=torch.int32)
        o = Opts(int(corr_path), None)
        self._chk(lib().fastncc_register_pair_host(
            self.h, C.c_void_p(ref.data_ptr()), ref.shape[0], ref.shape[1], C.c_void_p(sen.data_ptr()), sen.shape[0],
            sen.shape[1], C.c_void_p(points.data_ptr()), n, int(template_size), int(search_radius),
            C.byref(p) if p is not None else None, C.byref(o), C.c_void_p(raw.data_ptr())))
        return raw

    def sfoc_build_batch(self, images, p: Params = None, outs=None):
        n = len(images)
        for i, im in enumerate(images):
            self._cuda(im, "images[%d]" % i, torch.float32)
        ptrs = (C.c_void_p * n)(*[im.data_ptr() for im in images])
        Hs = (C.c_int * n)(*[im.shape[0] for im in images])
        Ws = (C.c_int * n)(*[im.shape[1] for im in images])
        pitches = (C.c_size_t * n)(*[im.shape[1] for im in images])
        hs = (C.c_void_p * n)(*[(outs[i].handle if outs is not None else None) for i in range(n)])
        self._chk(lib().sfoc_build_batch(self.h, n, ptrs, Hs, Ws, pitches, C.byref(p) if p is not None else None, hs))
        res = []
        for i in range(n):
            if outs is not None and hs[i] == outs[i].handle:
                res.append(outs[i])
            else:
                res.append(Cube(self, hs[i]))
        return res

    def fastncc_match_batch(self, refs, sens, points, template_sizes, search_radii, corr_path=CORR_AUTO, outs=None):
        """One (n, 6) int32 result tensor per pair (filled in place when
        `outs` is given: a repeated call with the same tensors reuses the
        context's plan)."""
        n = len(refs)
        if not (len(sens) == len(points) == len(template_sizes) == len(search_radii) == n):
            raise ValueError("refs, sens, points, template_sizes and search_radii must have the same length")
        for i, pt in enumerate(points):
            self._cuda(pt, "points[%d]" % i, torch.int32)
            _check_shape(pt, "points[%d]" % i, (pt.shape[0], 2))
        if outs is None:
            outs = [torch.empty((p.shape[0], 6), dtype=torch.int32, device=self.device) for p in points]
        else:
            for i, o in enumerate(outs):
                self._cuda(o, "outs[%d]" % i, torch.int32)
                _check_shape(o, "outs[%d]" % i, (points[i].shape[0], 6))
        R = (C.c_void_p * n)(*[c.handle for c in refs])
        S = (C.c_void_p * n)(*[c.handle for c in sens])
        Pp = (C.c_void_p * n)(*[p.data_ptr() for p in points])
        Np = (C.c_int * n)(*[p.shape[0] for p in points])
        Mp = (C.c_int * n)(*[int(v) for v in template_sizes])
        Rp = (C.c_int * n)(*[int(v) for v in search_radii])
        Op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        o = Opts(int(corr_path), None)
        self._chk(lib().fastncc_match_batch(self.h, n, R, S, Pp, Np, Mp, Rp, C.byref(o), Op))
        return outs

    def register_batch(self, refs, sens, points, template_sizes, search_radii, p: Params = None,
                       corr_path=CORR_AUTO, outs=None):
        """The whole path for a batch of pairs (fastncc_register_batch): lists
        of dense float32 device images and int32 (n, 2) device points; returns
        (or fills) one (n, 6) int32 result tensor per pair.  The first call
        with given tensors builds and captures the batch's plan; later calls
        with the same tensors replay it."""
        n = len(refs)
        if not (len(sens) == len(points) == len(template_sizes) == len(search_radii) == n):
            raise ValueError("refs, sens, points, template_sizes and search_radii must have the same length")
        for i in range(n):
            self._cuda(refs[i], "refs[%d]" % i, torch.float32)
            self._cuda(sens[i], "sens[%d]" % i, torch.float32)
            self._cuda(points[i], "points[%d]" % i, torch.int32)
            _check_shape(points[i], "points[%d]" % i, (points[i].shape[0], 2))
            if refs[i].dim() != 2 or sens[i].dim() != 2:
                raise ValueError("images must be 2-D")
        if outs is None:
            outs = [torch.empty((pt.shape[0], 6), dtype=torch.int32, device=self.device) for pt in points]
        else:
            for i, o in enumerate(outs):
                self._cuda(o, "outs[%d]" % i, torch.int32)
                _check_shape(o, "outs[%d]" % i, (points[i].shape[0], 6))
        o = Opts(int(corr_path), None)
        self._chk(lib().fastncc_register_batch(
            self.h, n, (C.c_void_p * n)(*[t.data_ptr() for t in refs]), (C.c_int * n)(*[t.shape[0] for t in refs]),
            (C.c_int * n)(*[t.shape[1] for t in refs]), (C.c_void_p * n)(*[t.data_ptr() for t in sens]),
            (C.c_int * n)(*[t.shape[0] for t in sens]), (C.c_int * n)(*[t.shape[1] for t in sens]),
            (C.c_void_p * n)(*[t.data_ptr() for t in points]), (C.c_int * n)(*[t.shape[0] for t in points]),
            (C.c_int * n)(*[int(v) for v in template_sizes]), (C.c_int * n)(*[int(v) for v in search_radii]),
            C.byref(p) if p is not None else None, C.byref(o), (C.c_void_p * n)(*[t.data_ptr() for t in outs])))
        return outs

    def _host_batch_args(self, refs, sens, points, template_sizes, search_radii, p, corr_path, outs):
        """The C arguments of the host-buffer batch calls (after the context),
        and the result tensors."""
        n = len(refs)
        if not (len(sens) == len(points) == len(template_sizes) == len(search_radii) == n):
            raise ValueError("refs, sens, points, template_sizes and search_radii must have the same length")
        for i in range(n):
            _check_host(refs[i], "refs[%d]" % i, torch.float32)
            _check_host(sens[i], "sens[%d]" % i, torch.float32)
            _check_host(points[i], "points[%d]" % i, torch.int32)
            _check_shape(points[i], "points[%d]" % i, (points[i].shape[0], 2))
            if refs[i].dim() != 2 or sens[i].dim() != 2:
                raise ValueError("images must be 2-D")
        if outs is None:
            outs = [torch.empty((pt.shape[0], 6), dtype=torch.int32) for pt in points]
        else:
            for i, o in enumerate(outs):
                _check_host(o, "outs[%d]" % i, torch.int32)
                _check_shape(o, "outs[%d]" % i, (points[i].shape[0], 6))
        o = Opts(int(corr_path), None)
        args = (n, (C.c_void_p * n)(*[t.data_ptr() for t in refs]), (C.c_int * n)(*[t.shape[0] for t in refs]),
                (C.c_int * n)(*[t.shape[1] for t in refs]), (C.c_void_p * n)(*[t.data_ptr() for t in sens]),
                (C.c_int * n)(*[t.shape[0] for t in sens]), (C.c_int * n)(*[t.shape[1] for t in sens]),
                (C.c_void_p * n)(*[t.data_ptr() for t in points]), (C.c_int * n)(*[t.shape[0] for t in points]),
                (C.c_int * n)(*[int(v) for v in template_sizes]), (C.c_int * n)(*[int(v) for v in search_radii]),
                C.byref(p) if p is not None else None, C.byref(o),
                (C.c_void_p * n)(*[t.data_ptr() for t in outs]))
        return args, outs

    def register_batch_host(self, refs, sens, points, template_sizes, search_radii, p: Params = None,
                            corr_path=CORR_AUTO, outs=None):
        """fastncc_register_batch_host: host (ideally pinned) tensors in,
        host result tensors out (synchronous)."""
        args, outs = self._host_batch_args(refs, sens, points, template_sizes, search_radii, p, corr_path, outs)
        self._chk(lib().fastncc_register_batch_host(self.h, *args))
        return outs

    def submit_batch_host(self, refs, sens, points, template_sizes, search_radii, p: Params = None,
                          corr_path=CORR_AUTO, outs=None):
        """fastncc_submit_batch_host: enqueues the batch and returns
        (ticket, outs) without waiting; the tensors are held until
        wait_batch_host(ticket), and outs are valid only after it."""
        args, outs = self._host_batch_args(refs, sens, points, template_sizes, search_radii, p, corr_path, outs)
        t = C.c_int64()
        self._chk(lib().fastncc_submit_batch_host(self.h, *args, C.byref(t)))
        if t.value:
            if not hasattr(self, "_held"):
                self._held = {}
            self._held[t.value] = (list(refs), list(sens), list(points), outs)
        return t.value, outs

    def wait_batch_host(self, ticket):
        """fastncc_wait_batch_host: blocks until the submission's results are
        in its outs; releases the tensors held for it (and for every earlier
        submission, which ends before it)."""
        self._chk(lib().fastncc_wait_batch_host(self.h, int(ticket)))
        held = getattr(self, "_held", {})
        for k in [k for k in held if k <= ticket]:
            del held[k]

    @property
    def plan_count(self) -> int:
        return int(lib().sfoc_ctx_plan_count(self.h))

    def plan_info(self):
        """The most recently used batch plan (sfoc_ctx_plan_info) as a dict."""
        import json
        n = C.c_size_t()
        self._chk(lib().sfoc_ctx_plan_info(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._chk(lib().sfoc_ctx_plan_info(self.h, buf, n.value, C.byref(n)))
        return json.loads(buf.value.decode())

    def stage_scopes(self, stage):
        """Milliseconds of each timed scope of a stage (by name) since the last reset."""
        idx = self.STAGES.index(stage)
        n = C.c_int()
        self._chk(lib().sfoc_ctx_stage_scopes(self.h, idx, None, 0, C.byref(n)))
        arr = (C.c_float * max(1, n.value))()
        self._chk(lib().sfoc_ctx_stage_scopes(self.h, idx, arr, n.value, C.byref(n)))
        return [float(arr[i]) for i in range(n.value)]

    def release_plans(self):
        self._chk(lib().sfoc_ctx_release_plans(self.h))

    def set_autotune(self, on=True):
        self._chk(lib().sfoc_ctx_set_autotune(self.h, 1 if on else 0))

    def autotune_entry(self, dtype, m, R, family=0):
        """{path, option, sample, candidates: [(path, option, ms)]} of the
        autotuner's entry for (dtype, m, R) in a family (0: AUTO, every form;
        1: IGEMM_TC, the tensor-core forms), or None."""
        path, opt, nc, smp = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        cp, co, cm = (C.c_int * 6)(), (C.c_int * 6)(), (C.c_float * 6)()
        self._chk(lib().sfoc_ctx_autotune_entry(self.h, int(dtype), int(m), int(R), int(family), C.byref(path),
                                                 C.byref(opt), C.byref(nc), cp, co, cm, C.byref(smp)))
        if path.value < 0:
            return None
        return dict(path=path.value, option=opt.value, sample=smp.value,
                    candidates=[(cp[i], co[i], float(cm[i])) for i in range(nc.value)])

    def autotune_export(self) -> str:
        n = C.c_size_t()
        self._chk(lib().sfoc_ctx_autotune_export(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._chk(lib().sfoc_ctx_autotune_export(self.h, buf, n.value, C.byref(n)))
        return buf.value.decode()

    def autotune_import(self, text: str):
        self._chk(lib().sfoc_ctx_autotune_import(self.h, text.encode()))

    def fast_blocks(self, image: torch.Tensor, threshold=0.05, grid_y=32, grid_x=32, margin=3):
        """Block-based FAST: (points (grid_y * grid_x, 2) int32 (x, y; -1 for
        an empty block), scores float32) on the device."""
        self._cuda(image, "image", torch.float32)
        H, W = image.shape
        nb = int(grid_y) * int(grid_x)
        pts = torch.empty((nb, 2), dtype=torch.int32, device=self.device)
        sc = torch.empty((nb,), dtype=torch.float32, device=self.device)
        self._chk(lib().sfoc_fast_blocks(self.h, _ptr(image), H, W, W, C.c_float(threshold), int(grid_y),
                                         int(grid_x), int(margin), _ptr(pts), _ptr(sc)))
        return pts, sc

    def rectify(self, image: torch.Tensor, model: torch.Tensor, out_shape=None, fill=0.0, out=None):
        """The sensed image resampled into the reference frame with the
        (3, 3) float64 device model (sensed -> reference), bilinear."""
        self._cuda(image, "image", torch.float32)
        self._cuda(model, "model", torch.float64)
        _check_shape(model, "model", (3, 3))
        H, W = image.shape
        oh, ow = out_shape or (H, W)
        if out is None:
            out = torch.empty((oh, ow), dtype=torch.float32, device=self.device)
        else:
            self._cuda(out, "out", torch.float32)
            _check_shape(out, "out", (oh, ow))
        self._chk(lib().sfoc_rectify(self.h, _ptr(image), H, W, W, _ptr(model), C.c_float(fill), oh, ow, _ptr(out)))
        return out

    def points_from_results(self, points: torch.Tensor, raw: torch.Tensor):
        """Control-point pairs of a match: (src, dst) float64 (n, 2) and the
        uint8 valid flags (status OK)."""
        self._cuda(points, "points", torch.int32)
        self._cuda(raw, "results", torch.int32)
        n = points.shape[0]
        _check_shape(points, "points", (n, 2))
        _check_shape(raw, "results", (n, 6))
        src = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        dst = torch.empty((n, 2), dtype=torch.float64, device=self.device)
        valid = torch.empty((n,), dtype=torch.uint8, device=self.device)
        self._chk(lib().fastncc_points_from_results(self.h, _ptr(points), _ptr(raw), n, _ptr(src), _ptr(dst),
                                                    _ptr(valid)))
        return src, dst, valid

    def fastncc_ransac(self, src: torch.Tensor, dst: torch.Tensor, samples: torch.Tensor, valid=None,
                       model=MODEL_PROJECTIVE, threshold=1.5, refits=1, want_scores=False):
        """RANSAC over src -> dst (float64 (n, 2) device tensors) with the
        given minimal samples (int32 (n_hyp, 4), or (n_hyp, 3) for the affine
        model).  Returns {H (3, 3) float64, inlier bool (n,), best, count,
        scores (n_hyp,) when asked} on the device (best/count as a tensor)."""
        self._cuda(src, "src", torch.float64)
        self._cuda(dst, "dst", torch.float64)
        self._cuda(samples, "samples", torch.int32)
        if valid is not None:
            self._cuda(valid, "valid", torch.uint8)
        n, n_hyp = src.shape[0], samples.shape[0]
        _check_shape(src, "src", (n, 2))
        _check_shape(dst, "dst", (n, 2))
        k = {MODEL_PROJECTIVE: 4, MODEL_AFFINE: 3}.get(int(model))
        if k is not None:  # an unknown model is refused by the library itself
            _check_shape(samples, "samples", (n_hyp, k))
        if valid is not None:
            _check_shape(valid, "valid", (n,))
        H = torch.empty((3, 3), dtype=torch.float64, device=self.device)
        inl = torch.empty((n,), dtype=torch.uint8, device=self.device)
        info = torch.empty((2,), dtype=torch.int32, device=self.device)
        sc = torch.empty((n_hyp,), dtype=torch.int32, device=self.device) if want_scores else None
        self._chk(lib().fastncc_ransac(self.h, _ptr(src), _ptr(dst), _ptr(valid) if valid is not None else None, n,
                                       int(model), _ptr(samples), n_hyp, float(threshold), int(refits), _ptr(H),
                                       _ptr(inl), _ptr(info), _ptr(sc) if sc is not None else None))
        out = dict(H=H, inlier=inl.bool(), info=info)
        if sc is not None:
            out["scores"] = sc
        return out


def results(raw: torch.Tensor):
    """Splits an (n, 6) int32 result buffer into named fields."""
    return _results(raw)


def workspace_bytes(n, R) -> int:
    return int(lib().sfoc_match_workspace_bytes(int(n), int(R)))
