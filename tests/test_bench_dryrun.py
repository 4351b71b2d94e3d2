"""bench.py's main flow on the CPU, with the library and the CUDA pieces of
torch replaced by stand-ins: the JSON line it assembles carries every key
the benchmark contract names, the fastest form heads it, and a failing
side measurement is reported in its own entry instead of costing the
line.  The numbers are the stand-ins' and mean nothing; the CPU baseline
runs the real oracle."""
import json
import sys
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402

STAGES = ("steer", "smooth", "integral", "template_stats", "correlation", "ncc_argmax", "other")
CORR_MS = {0: 0.8, 6: 0.8, 1: 7.5}     # auto (Fourier / tensor-core forms) and direct, per launch


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return 1e3 * (other.t - self.t) + 1e-3


def _fake_library(fail_ransac=False):
    b = types.SimpleNamespace()

    class SfocError(RuntimeError):
        def __init__(self, code, msg):
            super().__init__(msg)
            self.code = code

    b.SfocError = SfocError
    b.DTYPE_F32, b.DTYPE_BF16 = 0, 1
    b.CORR_AUTO, b.CORR_DIRECT_F32, b.CORR_IGEMM_TC, b.CORR_TC_BAND, b.CORR_TC_COLUMN, b.CORR_FFT = 0, 1, 2, 5, 4, 6
    b.params = lambda dtype=0, **kw: types.SimpleNamespace(dtype=dtype, cube_dtype=dtype)

    class Context:
        def __init__(self, device):
            self.launch_count = 0
            self.corr = 0
            self.n_steps = 0

        def _fill(self, pts, out):
            n = pts.shape[0]
            out.zero_()
            out[:, 5] = torch.where(torch.arange(n) % 10 == 9, 1, 0).to(torch.int32)

        def register_pair(self, d_ref, d_sen, d_pts, m, R, p=None, corr_path=0, out=None):
            self.corr = corr_path
            self.launch_count += 13
            self.n_steps += 1
            self._fill(d_pts, out)
            return out

        def register_pair_host(self, h_ref, h_sen, h_pts, m, R, p=None, corr_path=0, out=None):
            self._fill(h_pts, out)
            return out

        def sync(self):
            pass

        def measure_peaks(self):
            return {"fp32_tflops": 70.0, "fp32x2_tflops": 75.0, "fp64_tflops": 1.2, "hbm_copy_gbs": 6500.0}

        def autotune_entry(self, dtype, m, R, family=0):
            # F32 cubes: the Fourier form; BF16 cubes: the column form
            path, opt = (6, 128) if dtype == 0 else (4, 0)
            return {"path": path, "option": opt, "sample": 10, "candidates": [(path, opt, 0.5)]}

        def enable_timing(self, on=True):
            pass

        def reset_timing(self):
            self.n_steps = 0

        def stage_times(self):
            k = self.n_steps
            ms = {"steer": 0.18, "smooth": 0.6, "integral": 0.1, "template_stats": 0.04,
                  "correlation": CORR_MS.get(self.corr, 0.8), "ncc_argmax": 0.07, "other": 0.0}
            return {s: (ms[s] * k, k) for s in STAGES}

        def points_from_results(self, pts, raw):
            n = pts.shape[0]
            return (torch.zeros((n, 2), dtype=torch.float64), torch.zeros((n, 2), dtype=torch.float64),
                    torch.ones(n, dtype=torch.uint8))

        def fastncc_ransac(self, src, dst, samp, valid=None):
            if fail_ransac:
                raise SfocError(-4, "stand-in failure")
            return dict(H=torch.eye(3, dtype=torch.float64), inlier=torch.ones(src.shape[0], dtype=torch.bool),
                        info=torch.tensor([0, src.shape[0]], dtype=torch.int32))

        def rectify(self, img, H, out=None):
            return out

        def fast_blocks(self, img, t, gy, gx, margin):
            return torch.zeros((gy * gx, 2), dtype=torch.int32), torch.zeros(gy * gx)

        def sfoc_build(self, img, p=None, out=None):
            return out if out is not None else object()

        def fastncc_match(self, ref, sen, pts, m, R):
            raw = torch.zeros((pts.shape[0], 6), dtype=torch.int32)
            self._fill(pts, raw)
            return {"raw": raw}

    b.Context = Context
    pkg = types.ModuleType("paper_2202_13347_gb300")
    pkg.build = lambda *a, **k: None
    pkg.load = lambda: b
    return pkg


def _patch_cuda(monkeypatch):
    real_empty = torch.empty
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "set_device", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.Tensor, "cuda", lambda self, *a, **k: self)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)

    def empty(*a, device=None, **k):
        if a and isinstance(a[0], int) and a[0] >= 1 << 24:     # the 256 MB L2 flush buffer
            a = (1024,)
        return real_empty(*a, **k)

    monkeypatch.setattr(torch, "empty", empty)
    monkeypatch.setenv("PATH", "/nonexistent")                 # no nvidia-smi: empty clock samples


def _run(monkeypatch, capsys, argv, fail_ransac=False):
    import oracle
    oracle.build()        # compiled before PATH is blanked below (gcc is found through PATH)
    _patch_cuda(monkeypatch)
    monkeypatch.setitem(sys.modules, "paper_2202_13347_gb300", _fake_library(fail_ransac))
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    bench.main()
    out = capsys.readouterr().out.strip().splitlines()
    return json.loads(out[-1])


def test_line_has_every_contract_key(monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--workload", "inverting512", "--steps", "3", "--warmup", "3"])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["steps"] == 3 and line["warmup"] == 3 and line["n_gpus"] == 1 and line["scaling"] == "weak"
    assert "workload" in line["config"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in line["roofline"], k
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in line["cpu_baseline"], k
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] > 0
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in line["e2e"], k
    assert line["e2e"]["h2d_bytes_per_step"] > 0
    assert set(line["forms"]) == {"bf16", "f32", "f32direct"}
    # every form's results on the oracle's sampled points against the FP64 oracle
    for f in line["forms"]:
        par = line["forms"][f]["parity"]
        for k in ("points", "valid", "offsets_equal", "near_ties", "ncc_err_max_vs_fp64"):
            assert k in par, (f, k)
        assert par["points"] > 0
    best = max(line["forms"], key=lambda f: line["forms"][f]["value"])
    assert line["parity"] == line["forms"][best]["parity"]
    assert line["value"] == line["forms"][best]["value"] and line["config"]["form"] == best
    assert line["forms"]["f32direct"]["roofline"]["kernel"].startswith("k_corr_f32")
    assert line["gpu_launches"] == 13 * 3
    assert line["ransac"]["ms"] >= 0 and "roofline" in line["fast"]
    assert set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    # FP32 fractions use the measured peak (the faster FMA form), FAST one op per lane per clock
    assert line["forms"]["f32direct"]["roofline"]["peak"] == 75.0
    assert line["fast"]["roofline"]["peak"] == 35.0


def test_failing_side_measurement_keeps_the_line(monkeypatch, capsys):
    line = _run(monkeypatch, capsys, ["--workload", "inverting512", "--steps", "3", "--warmup", "3",
                                      "--no-cpu-baseline"], fail_ransac=True)
    assert "error" in line["ransac"] and line["match_quality"] is None
    assert line["value"] > 0 and "roofline" in line["fast"]


def test_reference_arm_line(monkeypatch, capsys):
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "inverting512",
                                      "--steps", "1", "--warmup", "1"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert np.isfinite(line["cpu_baseline"]["sfoc_mpix_s"])


def test_noise_sweep_line(monkeypatch, capsys):
    """--noise-sweep: one line with the CMR of every variant at every level
    of both noise series (Sec. 4.3)."""
    line = _run(monkeypatch, capsys, ["--noise-sweep"])
    assert line["template"] == 80 and line["pairs"] == 4
    assert set(line["cmr"]) == set(bench.NOISE_VARIANTS)
    assert set(line["sfoc_build_mpix_s"]) == set(bench.NOISE_VARIANTS)
    for v in line["cmr"].values():
        for kind, levels in bench.NOISE_LEVELS.items():
            assert len(v[kind]) == len(levels) and all(0.0 <= c <= 1.0 for c in v[kind])


def _fake_batch_library():
    pkg = _fake_library()
    b = pkg.load()
    base = b.Context

    class Context(base):
        def __init__(self, device):
            super().__init__(device)
            self.plans = 0

        def register_batch(self, refs, sens, pts, ms, Rs, p=None, corr_path=0, outs=None):
            self.plans = 1
            self.launch_count += 14
            self.n_steps += 1
            for pt, o in zip(pts, outs):
                self._fill(pt, o)
            return outs

        def register_batch_host(self, refs, sens, pts, ms, Rs, p=None, corr_path=0, outs=None):
            return self.register_batch(refs, sens, pts, ms, Rs, p, corr_path, outs)

        def submit_batch_host(self, refs, sens, pts, ms, Rs, p=None, corr_path=0, outs=None):
            self.tickets = getattr(self, "tickets", 0) + 1
            return self.tickets, self.register_batch(refs, sens, pts, ms, Rs, p, corr_path, outs)

        def wait_batch_host(self, ticket):
            assert 0 < ticket <= self.tickets

        def plan_info(self):
            return {"kind": 2, "graph": True, "classes": [{"path": 5, "cls": 3, "items": 10, "launches": 1,
                                                          "pairs": [0, 1]},
                                                         {"path": 6, "cls": 128, "items": 5, "launches": 1,
                                                          "pairs": [2]}]}

        def stage_scopes(self, stage):
            return [0.5, 0.2] if stage == "correlation" else []

        def autotune_entry(self, dtype, m, R, family=0):
            return {"path": 5, "option": 0, "sample": 10, "candidates": [(5, 0, 0.5), (4, 0, 0.7)]}

        def release_plans(self):
            self.plans = 0

        def fastncc_match(self, ref, sen, pts, m, R, corr_path=0):
            self.launch_count += 3
            return super().fastncc_match(ref, sen, pts, m, R)

    b.Context = Context
    return pkg


def test_batched_line(monkeypatch, capsys):
    """The default (batched) workload: the BF16-batched form heads the line,
    the plain FP32 form and the F32-batched form beside it, the roofline of
    the longest correlation class with every class listed, e2e through the
    host-buffer batch call, and the oracle sample's agreement."""
    from workloads import mixed_batch
    import oracle
    oracle.build()
    small = mixed_batch(seed=4100, n_pairs=3, scale=0.12)
    monkeypatch.setattr(bench, "batch_workload", lambda rank, workers, n_pairs=64, scale=1.0: (small, "3 small pairs"))
    _patch_cuda(monkeypatch)
    monkeypatch.setitem(sys.modules, "paper_2202_13347_gb300", _fake_batch_library())
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "3", "--warmup", "3"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert set(line["forms"]) == {"bf16batch", "f32batch", "f32plain"}
    assert line["config"]["form"] == "bf16batch" and line["value"] == line["forms"]["bf16batch"]["value"]
    assert line["dtype"] == "bf16" and line["scaling"] == "weak"
    roof = line["roofline"]
    assert roof["bound"] == "tensor" and len(roof["classes"]) == 2 and roof["launch_ms"] == 0.5
    assert line["e2e"]["h2d_bytes_per_step"] == sum(q.ref.nbytes + q.sen.nbytes + q.points.nbytes for q in small)
    # the timed steps are submissions, each waited for after the next one is in
    assert line["e2e"]["call"].startswith("fastncc_submit_batch_host") and len(line["e2e"]["step_done_ms"]) == 3
    assert line["e2e"]["results_equal_across_steps"] is True and len(line["e2e"]["sync_call_ms"]) == 3
    assert line["cpu_baseline"]["kind"] == "oracle" and line["parity"]["points"] > 0
    assert line["bf16batch_over_f32plain"] is not None
    assert line["gpu_launches"] == 14 * 3
    assert line["forms"]["bf16batch"]["autotune"]


def test_batched_reference_arm(monkeypatch, capsys):
    from workloads import mixed_batch
    small = mixed_batch(seed=4100, n_pairs=3, scale=0.12)
    monkeypatch.setattr(bench, "batch_workload", lambda rank, workers, n_pairs=64, scale=1.0: (small, "3 small pairs"))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"])
    bench.main()
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["d2h_bytes_per_step"] == 0
