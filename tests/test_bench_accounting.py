"""The work figures behind the benchmark's roofline numerators, against the
per-point numbers the design notes and profiles state, and the whole-job
throughput arithmetic.  No GPU needed."""
from types import SimpleNamespace

import pytest

import bench


def _pair(m, R):
    return SimpleNamespace(m=m, R=R)


@pytest.mark.parametrize("m,R,want", [(41, 10, 1.78e7), (81, 20, 2.647e8), (101, 40, 1.606e9)])
def test_direct_flop_per_point(m, R, want):
    """2 m^2 z (2R+1)^2 with z = 12 (Eq. 10 at every offset): the 512^2,
    2048^2 and 10000^2 workloads' template and search sizes."""
    assert bench.corr_flops(_pair(m, R)) == pytest.approx(want, rel=2e-3)


def test_fourier_flop_per_point():
    """The Fourier form's count for m = 81, R = 20 on 128-point transforms:
    15.06 Mflop per point, the figure its profile summary quotes."""
    p = _pair(81, 20)
    assert bench.fft_side(p) == 128
    assert bench.fft_flops(p) == pytest.approx(15.0592e6, rel=1e-5)
    assert bench.fft_side(_pair(41, 10)) == 64
    assert bench.fft_side(_pair(101, 40)) is None      # m + 2R = 181 > 128: no Fourier form


def test_job_value():
    """934 matched points per step, 20 steps in 35.95 ms: 519.6 K CP/s."""
    assert bench.job_value(934, 20, 35.95) == pytest.approx(519610.6, rel=1e-6)
    assert bench.reduce_over_ranks(None, None, 12.5, 7, "cpu") == (12.5, 7)


def test_clock_sampler_keeps_the_timed_region(tmp_path, monkeypatch):
    """The clocks object describes the timed region: samples before it (an
    idle GPU during host-side set-up) are left out, the first sample after a
    short region is waited for and kept, throttle reasons are reported."""
    import os
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/bash\nsleep 0.2\ni=0\nwhile true; do\n"
                    "  if [ $i -lt 3 ]; then c=990; r='Not Active'; else c=2070; r='Active'; fi\n"
                    "  echo \"0, $c, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, $r\"\n"
                    "  i=$((i+1)); sleep 0.2\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as cs:
        assert cs.lines                          # running before the region starts
        time.sleep(0.45)
        t0 = time.monotonic()
        time.sleep(0.03)
        t1 = time.monotonic()
        cs.mark(t0, t1)
    s = cs.summary()
    assert s["sm_mhz"] == 2070.0 and s["scope"] == "timed region + one period"
    assert s["reasons"] == ["sw_power_cap"]
    # without nvidia-smi the line still gets a clocks object, with no samples
    monkeypatch.setenv("PATH", str(tmp_path / "nowhere"))
    with bench.ClockSampler(0) as cs2:
        cs2.mark(0.0, 0.0)
    assert cs2.summary()["samples"] == 0


def test_noise_series_are_the_papers():
    """The sweep's variances and template size are the ones Sec. 4.3 prints
    (tests/golden/paper_values.txt)."""
    import os
    vals = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            vals[k] = v
    for kind, vmax, step in (("gaussian", "gauss_var_max", "gauss_var_step"),
                             ("speckle", "speckle_var_max", "speckle_var_step")):
        lv = bench.NOISE_LEVELS[kind]
        assert lv[0] == 0 and lv[-1] == pytest.approx(float(vals[vmax]))
        assert all(b - a == pytest.approx(float(vals[step])) for a, b in zip(lv, lv[1:]))
    assert bench.NOISE_TEMPLATE == int(vals["noise_template"])


def test_form_rooflines_reproduce_the_last_line():
    """form_roofline against the figures of a GB300 run of the 2048^2
    workload (999 processed points, the measured bf16 peak 1921.3 TFLOP/s),
    for the concrete form each step ran: 0.79 ms per Fourier launch (on F32
    or BF16 cubes: the same transform count), 1.1598 ms per column-form
    launch, 7.51 ms per direct launch."""
    p = _pair(81, 20)
    pk = {"bf16": 1921.3, "src": "measured"}
    f = bench.form_roofline("f32", p, 0.79, 999, pk, "sar2048", 6, 128)
    assert f["bound"] == "alu" and f["kernel"].startswith("k_corr_fft<128>") and "F32 cubes" in f["kernel"]
    assert f["achieved"] == pytest.approx(19.04, rel=2e-3) and f["frac"] == pytest.approx(0.2364, rel=2e-3)
    assert f["traffic"] is None  # no capture of the kernel as it stands
    fb = bench.form_roofline("bf16", p, 0.79, 999, pk, "sar2048", 6, 0)
    assert fb["bound"] == "alu" and "BF16 cubes" in fb["kernel"] and fb["achieved"] == pytest.approx(19.04, rel=2e-3)
    t = bench.form_roofline("bf16", p, 1.1598, 999, pk, "sar2048", 4)
    assert t["bound"] == "tensor" and t["kernel"].startswith("k_corr_tc_col")
    assert t["achieved"] == pytest.approx(228.0, rel=2e-3) and t["traffic"] is None
    bb = bench.form_roofline("bf16", p, 1.1598, 999, pk, "sar2048", 5)
    assert bb["kernel"].startswith("k_corr_tc_band")
    assert bb["traffic"] == pytest.approx(91.73e6 / 304 * 999, rel=1e-3)  # the capture's bytes per point x points
    d = bench.form_roofline("f32direct", p, 7.51, 999, pk, "sar2048", 1)
    assert d["kernel"].startswith("k_corr_f32") and d["achieved"] == pytest.approx(35.2, rel=5e-3)
    assert d["traffic"] is None


def test_fast_roofline():
    """Block FAST on a 2048^2 image in 0.0843 ms (a GB300 run): 179 FP32 ops
    per pixel give 8.9 Top/s, 22 % of 40.3 Top/s; the image read is 199 GB/s."""
    assert bench.FAST_OPS_PER_PX == 179
    r = bench.fast_roofline(0.0843, 2048, 2048, 6780.0)
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(40.28, rel=1e-3)
    assert r["achieved"] == pytest.approx(8.906, rel=2e-3) and r["frac"] == pytest.approx(0.2211, rel=3e-3)
    assert r["hbm_gbs"] == pytest.approx(199.0, rel=2e-3)


def test_batch_roofline_scales_the_band_capture_to_a_class():
    """The batched line's `traffic`: a band-form class of one template side
    with a capture of its instance gets the capture's bytes per processed
    point times the class's processed points (per launch); classes of other
    sizes, or of several template sides, get none."""
    pairs = [_pair(101, 40), _pair(101, 35), _pair(81, 20)]
    info = {"classes": [{"path": 5, "cls": 6, "launches": 1, "pairs": [0, 1], "items": 30},
                        {"path": 5, "cls": 4, "launches": 1, "pairs": [2], "items": 10}]}
    r = {"info": info, "scopes": [20.0, 2.0], "processed": [20, 10, 10]}
    pk = {"bf16": 1957.5, "bf16_sus": 1761.3, "src": "measured"}
    line = bench.batch_roofline("bf16batch", pairs, r, pk)
    per_pt = bench.BAND_TRAFFIC_PER_POINT[(101, 6)]
    assert per_pt == pytest.approx(789.52e6 / 851, rel=1e-4)
    assert line["kernel"].endswith("class 6") and line["traffic"] == pytest.approx(per_pt * 30)
    small = [c for c in line["classes"] if c["cls"] == 4][0]
    assert small["traffic"] is None and small["m"] == [81] and small["R"] == [20, 20]
