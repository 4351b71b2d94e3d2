"""The C-ABI library builds, loads without a GPU and exports every entry
point include/sfoc.h declares; struct layouts agree between C and the
binding; host-only calls behave.  No compute call runs here."""
import ctypes as C
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        names |= set(re.findall(r"^SFOC_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def b():
    import paper_2202_13347_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(b):
    names = declared()
    assert len(names) >= 19
    L = C.CDLL(b.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # and the binding knows every one of them
    assert names <= set(b._SIGS), names - set(b._SIGS)


def test_struct_layouts_match_c(b, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sfoc.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(sfoc_params), sizeof(fastncc_result),'
        ' sizeof(fastncc_opts), offsetof(sfoc_params, cube_dtype), offsetof(fastncc_result, status),'
        ' offsetof(fastncc_opts, d_maps)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [C.sizeof(b.Params), C.sizeof(b.Result), C.sizeof(b.Opts), b.Params.cube_dtype.offset,
                    b.Result.status.offset, b.Opts.d_maps.offset]


def test_params_default_are_the_paper_values(b):
    p = b.Params()
    assert b.lib().sfoc_params_default(C.byref(p)) == 0
    assert [p.scales[i] for i in range(p.n_scales)] == [0.6, 0.8, 1.0]      # Table 2
    assert p.sigma2 == 1.5 and p.n_orient == 6                                # Table 2, Sec. 2.1
    assert [p.dil[i] for i in range(p.n_dil)] == [1, 2, 3]                    # Sec. 2.1
    assert p.rectify == 1 and p.radius_mult == 3.0 and p.cube_dtype == 0
    assert b.lib().sfoc_params_default(None) == -1


def test_host_only_calls(b):
    L = b.lib()
    assert L.sfoc_match_workspace_bytes(-1, 3) == 0
    assert L.sfoc_match_workspace_bytes(10, 2) > 10 * 25 * 4
    assert L.sfoc_ctx_destroy(None) == -1
    assert L.sfoc_cube_free(None) == -1
    assert L.sfoc_last_error_string(None) == b"null context"
    assert L.sfoc_build(None, None, 1, 1, 1, None, 0, 0, None, None) == -1
    assert L.fastncc_match(None, None, None, None, 0, 1, 1, None, None) == -1


def test_null_context_is_rejected_everywhere(b):
    """Every entry point that takes a context (or a cube) refuses a NULL
    one with SFOC_ERR_INVALID_ARG before touching the device, whatever the
    other arguments are (here all zero / NULL)."""
    L = b.lib()
    host_only = {"sfoc_ctx_create", "sfoc_match_workspace_bytes", "sfoc_params_default", "sfoc_last_error_string",
                 "sfoc_ctx_launch_count", "sfoc_ctx_plan_count"}
    checked = 0
    for name, (res, args) in b._SIGS.items():
        if name in host_only:
            continue
        vals = [0.0 if a in (C.c_float, C.c_double) else (0 if a in (C.c_int, C.c_size_t, C.c_int64) else None)
                for a in args]
        assert getattr(L, name)(*vals) == -1, name
        checked += 1
    assert checked >= 24
    assert L.sfoc_ctx_launch_count(None) == 0 and L.sfoc_ctx_plan_count(None) == 0
    assert L.sfoc_ctx_create(None, 0, None) == -1


def test_context_without_a_device():
    """Without a reachable CUDA device sfoc_ctx_create reports SFOC_ERR_CUDA
    and leaves *out NULL (an out-of-range index is SFOC_ERR_INVALID_ARG)."""
    torch = pytest.importorskip("torch")
    import paper_2202_13347_gb300 as pkg
    pkg.build()
    b = pkg.load()
    L = b.lib()
    h = C.c_void_p(1)
    if torch.cuda.is_available():
        assert L.sfoc_ctx_create(C.byref(h), 1 << 20, None) == -1 and h.value is None
        pytest.skip("a CUDA device is present")
    assert L.sfoc_ctx_create(C.byref(h), 0, None) == -4
    assert h.value is None

def test_no_oracle_in_product_path():
    """The product package never imports the oracle and the library holds no
    CPU fallback: the sources do not mention it."""
    pkg = os.path.join(ROOT, "paper_2202_13347_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "liboracle" not in txt, f


def test_binding_shape_checks(b):
    """The binding checks every tensor's shape and dtype against the sizes
    it passes, since the library reads and writes exactly those sizes."""
    torch = pytest.importorskip("torch")
    b._check_shape(torch.zeros((3, 2)), "x", (3, 2))
    with pytest.raises(ValueError):
        b._check_shape(torch.zeros((6,)), "x", (3, 2))
    with pytest.raises(ValueError):
        b._check_shape(torch.zeros((3, 3)), "x", (3, 2))
    assert b._channels(None) == 12
    assert b._channels(b.params(n_orient=8, first_order_only=True)) == 8
    assert b._channels(b.params(n_orient=4)) == 8
    b._check_host(torch.zeros(3, dtype=torch.float32), "h", torch.float32)
    with pytest.raises(ValueError):
        b._check_host(torch.zeros(3, dtype=torch.float64), "h", torch.float32)
    with pytest.raises(ValueError):
        b._check_host(torch.zeros((4, 4), dtype=torch.float32).t(), "h", torch.float32)


def test_submitted_batch_keeps_its_tensors_until_waited(b, monkeypatch):
    """submit_batch_host hands the library raw pointers and returns at once,
    so the binding holds each submission's tensors until wait_batch_host
    returns for its ticket or a later one; the pointers and shapes passed are
    the tensors' own.  (The library is stubbed: no device.)"""
    import torch
    seen = []

    class Stub:
        def fastncc_submit_batch_host(self, h, n, refs, Hr, Wr, sens, Hs, Ws, pts, npts, ms, Rs, p, o, outs, t):
            seen.append((n, [refs[i] for i in range(n)], [Hr[i] for i in range(n)], [Ws[i] for i in range(n)],
                         [npts[i] for i in range(n)], [ms[i] for i in range(n)], o._obj.corr_path))
            t._obj.value = len(seen)
            return 0

        def fastncc_wait_batch_host(self, h, t):
            return 0 if 0 <= t <= len(seen) else -1

        def sfoc_last_error_string(self, h):
            return b"unknown batch ticket"

    monkeypatch.setattr(b, "lib", lambda: Stub())
    ctx = object.__new__(b.Context)
    ctx.h, ctx.device = C.c_void_p(1), torch.device("cuda", 0)
    try:
        refs = [torch.zeros((30, 40)), torch.zeros((50, 20))]
        sens = [torch.zeros((31, 41)), torch.zeros((51, 21))]
        pts = [torch.zeros((3, 2), dtype=torch.int32), torch.zeros((5, 2), dtype=torch.int32)]
        t1, o1 = ctx.submit_batch_host(refs, sens, pts, [9, 11], [2, 3], corr_path=b.CORR_TC_BAND)
        t2, o2 = ctx.submit_batch_host(refs, sens, pts, [9, 11], [2, 3])
        assert (t1, t2) == (1, 2)
        assert [tuple(o.shape) for o in o1] == [(3, 6), (5, 6)]
        n, ptr, H, W, npt, m, corr = seen[0]
        assert n == 2 and ptr == [r.data_ptr() for r in refs] and H == [30, 50] and W == [41, 21]
        assert npt == [3, 5] and m == [9, 11] and corr == b.CORR_TC_BAND
        assert set(ctx._held) == {1, 2} and ctx._held[1][3] is o1
        ctx.wait_batch_host(1)
        assert set(ctx._held) == {2}
        ctx.wait_batch_host(2)
        assert not ctx._held
        with pytest.raises(b.SfocError):
            ctx.wait_batch_host(7)
        with pytest.raises(ValueError):  # images must be float32
            ctx.submit_batch_host([torch.zeros((3, 3), dtype=torch.float64)], sens[:1], pts[:1], [1], [0])
    finally:
        ctx.h = None  # nothing to destroy: the handle is the stub's
