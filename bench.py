#!/usr/bin/env python
"""Benchmark of the fine-registration hot path of arXiv 2202.13347 on GB300.

One step = the whole path on one batch of synthetic image pairs: SFOC cube
of every reference and sensed image (Sec. 2.1), the integral images of the
searched cubes, template statistics, correlation R_ST, NCC (Eq. 9), argmax
and sub-pixel refinement for every interest point (Sec. 2.2, Sec. 3.2.2).

Default workload (--workload mixed64): 64 seeded pairs of uneven size
(sides 512-4096, non-square), each with its own radiometric map, 200-4000
block points, template from {41, 61, 81, 101} and search radius in
[10, 40]; 12 SFOC channels.  Forms:
  bf16batch  BF16 cubes, every pair in one batched launch per stage, the
             correlation form of each (m, R) measured by the autotuner
             (tensor-core forms), the whole step a replayed CUDA graph:
             the line's value;
  f32batch   the same with F32 cubes (Fourier or direct FP32 correlation);
  f32plain   F32 cubes, the direct FP32 correlation, pairs one after the
             other (the plain FP32 GPU form).
The single-pair workloads (--workload sar2048: 2048^2 optical-like vs
SAR-like, 1000 points, m=81, R=20; inverting512; speckle10000) time the
forms bf16 (tensor cores), f32 (Fourier where it runs) and f32direct.

Metric: matched control points per second (points whose status is OK),
whole job over all ranks; SFOC Mpix/s is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload mixed64|sar2048|inverting512|speckle10000]
Under torchrun each rank runs its own shard of the job (its own seeded
batch or pair: weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "matched CPs/sec and SFOC Mpix/sec on 1 GB300, BF16-batched vs plain FP32"
UNIT = "CP/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
FFT_SIZES = (64, 128)  # transform sides of the Fourier correlation (the smallest with m + 2R <= L)
# DRAM bytes (read + write) per processed point of a correlation kernel on
# the 2048x2048 workload (m = 81, R = 20), keyed by (form, correlation path),
# from one ncu capture of the kernel as it stands (the band form: 87.12 MB
# read + 4.61 MB written for the autotuner's 304-point launch); absent where
# none is current.  A launch's traffic is this times the points it processed.
CORR_TRAFFIC_PER_POINT_SAR2048 = {("bf16", 5): (87.118848e6 + 4.611072e6) / 304}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed64", choices=["mixed64", "inverting512", "sar2048", "speckle10000"])
    ap.add_argument("--forms", default=None,
                    help="mixed64: bf16batch,f32batch,f32plain; single pairs: bf16 (BF16 cubes, tensor-core "
                         "correlation), f32 (F32 cubes, automatic correlation), f32direct (F32 cubes, the plain "
                         "direct correlation)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="mixed64 under torchrun: weak = every rank its own seeded 64-pair batch (its shard of a "
                         "64 x N-pair job); strong = one 64-pair job whose pairs are balanced over the ranks by "
                         "cost, results gathered on rank 0")
    ap.add_argument("--corr", default="auto", choices=["auto", "igemm_tc", "band", "column", "fft", "direct"],
                    help="correlation path of the batched forms and of the single-pair bf16 / f32 forms (auto: "
                         "the autotuner's measured choice)")
    ap.add_argument("--template", type=int, default=0,
                    help="single-pair workloads: template side m instead of the workload's (profiling cases)")
    ap.add_argument("--radius", type=int, default=-1,
                    help="single-pair workloads: search radius R instead of the workload's (profiling cases)")
    ap.add_argument("--pairs", type=int, default=64, help="mixed64: pairs per batch (fewer for small profiling cases)")
    ap.add_argument("--scale", type=float, default=1.0, help="mixed64: side and point-count scale (1 = full size)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--noise-sweep", action="store_true",
                    help="instead of the benchmark: CMR of the descriptor variants under the noise series of Sec. 4.3")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return dict(hbm=float(d["hbm_gbs"]), bf16=float(d["bf16_tflops"]),
                    bf16_sus=float(d.get("bf16_tflops_sustained", d["bf16_tflops"])), src="measured")
    except Exception:
        return dict(hbm=6800.0, bf16=1900.0, bf16_sus=1700.0, src="fallback")


def workload(name, rank):
    from workloads import inverting_pair_512, sar_pair_2048, speckle_pair_10000
    if name == "inverting512":
        p = inverting_pair_512(seed=1000 + 7919 * rank)
        desc = "512x512 pair, piecewise inverting map, 100 block-max points, m=41, R=10, z=12"
    elif name == "speckle10000":
        p = speckle_pair_10000(seed=5000 + 7919 * rank)
        desc = ("10000x10000 uint16 reference (read as v/65535) vs L=1 speckled sensed image under block affine "
                "residuals, 10000 points, m=101, R=40, z=12")
    else:
        p = sar_pair_2048(seed=2000 + 7919 * rank)
        desc = ("2048x2048 optical-like ref vs SAR-like sensed (Gamma L=4 speckle, 256-px shift field), "
                "1000 block-Harris points, m=81, R=20, z=12")
    return p, desc


def batch_workload(rank, workers, n_pairs=64, scale=1.0):
    """The mixed batch of this rank (its own seed: under torchrun each
    rank's batch is its shard of a 64 x N-pair job)."""
    from workloads import mixed_batch
    pairs = mixed_batch(seed=4000 + 7919 * rank, n_pairs=n_pairs, scale=scale, workers=workers)
    px = sum(q.ref.size + q.sen.size for q in pairs)
    pts = sum(len(q.points) for q in pairs)
    desc = ("%d pairs, sides U[512,4096]%s (non-square), linear/gamma/inverted/speckled maps, 200-4000%s block "
            "points, m in {41,61,81,101}, R in U[10,40], z=12: %d points, %.1f Mpx"
            % (n_pairs, "" if scale == 1.0 else " x %g" % scale, "" if scale == 1.0 else " x %g" % scale, pts,
               px / 1e6))
    return pairs, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    Samples are time-stamped as they arrive.  After `mark(t0, t1)` (the
    timed region, time.monotonic()), the summary keeps the samples taken in
    it and in the sampling period after it (up to 1.5 periods, for jitter:
    a region of a few tens of ms holds no 200 ms sample of its own), and
    __exit__ waits (bounded) for that sample.  Without a mark, or with no sample there, every sample
    of the run counts."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    PERIOD = 0.2  # seconds between samples (-lms 200)

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.lines = []       # (arrival time, csv line)
        self.proc = None
        self.window = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi can take longer to print its first sample than a short
            # timed region lasts: wait (bounded) until it is running
            t0 = time.monotonic()
            while not self.lines and self.proc.poll() is None and time.monotonic() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            if self.window is not None:
                t_end = self.window[1]
                while (not any(ts > t_end for ts, _ in self.lines) and self.proc.poll() is None
                       and time.monotonic() - t_end < 3 * self.PERIOD):
                    time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        lines = list(self.lines)
        scope = "run"
        if self.window is not None:
            t0, t1 = self.window
            near = [(ts, ln) for ts, ln in lines if t0 <= ts <= t1 + 1.5 * self.PERIOD]
            if near:
                lines, scope = near, "timed region + one period"
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "scope": scope}


def run_form(b, torch, ctx, pair, form, steps, warmup, flush, corr_name="auto"):
    p = b.params(dtype=b.DTYPE_BF16 if form == "bf16" else b.DTYPE_F32)
    corr = b.CORR_DIRECT_F32 if form == "f32direct" else corr_option(b, corr_name)
    d_ref = torch.from_numpy(pair.ref).cuda()
    d_sen = torch.from_numpy(pair.sen).cuda()
    d_pts = torch.from_numpy(pair.points).cuda()
    raw = torch.empty((len(pair.points), 6), dtype=torch.int32, device="cuda")

    def step():
        ctx.register_pair(d_ref, d_sen, d_pts, pair.m, pair.R, p=p, corr_path=corr, out=raw)

    for _ in range(warmup):
        step()
    ctx.sync()
    stream = torch.cuda.current_stream()
    ctx.enable_timing(True)
    ctx.reset_timing()
    l0 = ctx.launch_count
    evs = []
    torch.cuda.synchronize()
    t_start = time.monotonic()
    for _ in range(steps):
        flush.zero_()                       # L2 flush (256 MB write), outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    t_end = time.monotonic()
    launches = ctx.launch_count - l0
    ctx.sync()
    st = ctx.stage_times()
    ctx.enable_timing(False)
    ms = [a.elapsed_time(c) for a, c in evs]
    status = raw[:, 5].cpu()
    # the concrete correlation form the steps ran: the autotuner's entry for
    # an AUTO form, the forced form otherwise
    path, option = int(corr), 0
    if corr == b.CORR_AUTO:
        ent = ctx.autotune_entry(p.cube_dtype, pair.m, pair.R)
        if ent is not None:
            path, option = ent["path"], ent["option"]
    return dict(ms=sum(ms), ms_steps=ms, matched=int((status == 0).sum()), valid=int(((status == 0) | (status == 3)).sum()),
                stages=st, launches=launches, p=p, corr=corr, d=(d_ref, d_sen, d_pts), raw=raw,
                t_timed=(t_start, t_end), path=path, option=option)


# FP32 operations of one FAST-9 score as k_fast_blocks computes it: 16
# differences to the centre, 32 + 32 min/max for the windows of 2 and 4
# circle pixels (both polarities), 6 per arc for the 16 arcs of 9, 3 to
# finish
FAST_OPS_PER_PX = 16 + 32 + 32 + 16 * 6 + 3
FP32_OPS_PEAK = 152 * 128 * 2.070e9 / 1e12   # Top/s: one FP32 add / min / max per lane per clock


def fast_roofline(ms, H, W, hbm_gbs, pk=None):
    """Block FAST is bound by its score arithmetic, not by HBM (the image is
    read once, 4 B/px): achieved = FAST_OPS_PER_PX per pixel of the image
    over the launch time, against one FP32 op per lane per clock (half the
    measured scalar FMA flop rate, which counts 2 flop per FMA)."""
    ach = FAST_OPS_PER_PX * H * W / (ms * 1e-3) / 1e12
    gbs = 4.0 * H * W / (ms * 1e-3) / 1e9
    if pk and pk.get("fp32_scalar"):
        peak, src = pk["fp32_scalar"] / 2.0, "scalar FFMA chains of sfoc_measure_peaks, one op per lane per clock"
    else:
        peak, src = FP32_OPS_PEAK, "152 SMs x 128 FP32 lanes x 2070 MHz (nominal)"
    return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Top/s", "frac": ach / peak,
            "work": "%d FP32 ops per pixel (FAST-9 score by windowed min / max)" % FAST_OPS_PER_PX,
            "peak_src": src, "hbm_gbs": gbs, "hbm_frac": gbs / hbm_gbs}


def run_fast(torch, ctx, pair, hbm_gbs, reps=10, grid=32, t=0.05, pk=None):
    """Block-based FAST (Sec. 3.1.1) on the sensed image of the workload,
    timed apart from the step (CUDA events, median of reps)."""
    img = torch.from_numpy(pair.sen).cuda()
    margin = pair.m // 2 + pair.R
    for _ in range(2):
        pts, sc = ctx.fast_blocks(img, t, grid, grid, margin)
    stream = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.fast_blocks(img, t, grid, grid, margin)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    H, W = pair.sen.shape
    return dict(ms=ms, mpix_s=pair.sen.size / (ms * 1e-3) / 1e6, blocks=grid * grid,
                points=int((pts[:, 0] >= 0).sum()), threshold=t, margin=margin,
                roofline=fast_roofline(ms, H, W, hbm_gbs, pk), launches=1)


def run_ransac(b, torch, ctx, pair, r, n_hyp=4096, reps=10, seed=7):
    """The outlier rejection that follows matching (Sec. 3.2.3): projective
    RANSAC over the step's control points with n_hyp seeded minimal samples,
    timed apart from the step (CUDA events, median of reps); plus the
    matches' NCM / CMR / RMSE (Sec. 4.1) against the planted ground truth."""
    import numpy as np
    from workloads import ransac_samples
    d_pts, raw = r["d"][2], r["raw"]
    src, dst, valid = ctx.points_from_results(d_pts, raw)
    samp = torch.from_numpy(ransac_samples(seed, src.shape[0], n_hyp, 4)).cuda()
    for _ in range(2):
        g = ctx.fastncc_ransac(src, dst, samp, valid=valid)
    stream = torch.cuda.current_stream()
    t = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g = ctx.fastncc_ransac(src, dst, samp, valid=valid)
        e1.record(stream)
        e1.synchronize()
        t.append(e0.elapsed_time(e1))
    info = g["info"].cpu().numpy()
    # rectification of the sensed image with the fitted model (Sec. 3.2.3)
    img = torch.from_numpy(pair.sen).cuda()
    out = torch.empty_like(img)
    for _ in range(2):
        ctx.rectify(img, g["H"], out=out)
    tr = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.rectify(img, g["H"], out=out)
        e1.record(stream)
        e1.synchronize()
        tr.append(e0.elapsed_time(e1))
    rect_ms = statistics.median(tr)
    res = raw.cpu().numpy()
    ok = res[:, 5] == 0
    off = np.stack([res[:, 3].view(np.float32), res[:, 4].view(np.float32)], 1).astype(np.float64)  # refined offsets
    err = np.linalg.norm(off - pair.truth, axis=1)
    correct = ok & (err <= 1.5)
    ncm = int(correct.sum())
    quality = dict(ncm=ncm, cmr=ncm / max(1, int(ok.sum())),
                   rmse=float(np.sqrt(np.mean(err[correct] ** 2))) if ncm else None, tolerance_px=1.5,
                   truth="planted offset of each point")
    return dict(ms=statistics.median(t), hypotheses=n_hyp, points=int(src.shape[0]), valid=int(valid.sum()),
                inliers=int(info[1]), best_hypothesis=int(info[0]), model="projective", threshold_px=1.5,
                launches=3,
                rectify={"ms": rect_ms, "mpix_s": pair.sen.size / (rect_ms * 1e-3) / 1e6,
                         "gb_s": 8.0 * pair.sen.size / (rect_ms * 1e-3) / 1e9,
                         "work": "4 B read + 4 B written per output pixel (bilinear, FP64 mapping)"}), quality


def run_e2e(b, torch, ctx, pair, p, corr, steps):
    h_ref = torch.from_numpy(pair.ref).pin_memory()
    h_sen = torch.from_numpy(pair.sen).pin_memory()
    h_pts = torch.from_numpy(pair.points).pin_memory()
    out = torch.empty((len(pair.points), 6), dtype=torch.int32).pin_memory()
    ctx.register_pair_host(h_ref, h_sen, h_pts, pair.m, pair.R, p=p, corr_path=corr, out=out)
    t = []
    for _ in range(steps):
        t0 = time.perf_counter()
        ctx.register_pair_host(h_ref, h_sen, h_pts, pair.m, pair.R, p=p, corr_path=corr, out=out)
        t.append(time.perf_counter() - t0)
    matched = int((out[:, 5] == 0).sum())
    h2d = h_ref.numel() * 4 + h_sen.numel() * 4 + h_pts.numel() * 4
    d2h = out.numel() * 4
    return dict(ms=1e3 * sum(t), steps=steps, matched=matched, unit=UNIT, h2d_bytes_per_step=h2d,
                d2h_bytes_per_step=d2h)


def cpu_baseline(pair, n_sample=64, seed=99):
    """The oracle as it stands on a seeded sample of the workload's points
    (64: about 12 s on 16 host cores at m = 81, R = 20), plus its SFOC build
    rate on an image region."""
    import numpy as np
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pair.points), min(n_sample, len(pair.points)), replace=False))
    t0 = time.perf_counter()
    o = oracle.match_pair(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R)
    dt = time.perf_counter() - t0
    matched = int((o["status"] == 0).sum())
    mpix, region = oracle_sfoc_mpix(pair)
    cpu = dict(value=matched / dt, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
               sample="%d of %d points (seeded), FP64 SFOC on their windows only, Eq. 8 NCC" % (len(idx), len(pair.points)),
               seconds=dt, sfoc_mpix_s=mpix, sfoc_sample=region)
    return cpu, (idx, o)


def form_parity(raw, idx, o):
    """A form's results on the oracle's sampled points against the unrounded
    FP64 oracle: valid points, offsets equal, near ties (the oracle's
    best-vs-second margin <= 2e-4) and the largest NCC difference where the
    offsets agree."""
    import numpy as np
    g = raw.cpu().numpy()[idx]
    ok = np.isin(o["status"], [0, 3])
    same = ok & (g[:, 0] == o["dx"]) & (g[:, 1] == o["dy"])
    err = 0.0
    if same.any():
        gn = g[:, 2].view(np.float32).astype(np.float64)
        err = float(np.abs(gn[same] - o["ncc"][same]).max())
    return dict(points=int(len(idx)), valid=int(ok.sum()), offsets_equal=int(same.sum()),
                near_ties=int((ok & (o["margin"] <= 2e-4)).sum()), ncc_err_max_vs_fp64=err)


def oracle_sfoc_mpix(pair, side=512):
    """The oracle's SFOC build rate (Mpix/s) on a centred side x side region
    of the sensed image: all 12 channels in FP64, direct 2-D filtering."""
    import oracle
    H, W = pair.sen.shape
    side = min(side, H, W)
    y0, x0 = (H - side) // 2, (W - side) // 2
    t0 = time.perf_counter()
    oracle.sfoc_roi(pair.sen, None, y0, x0, side, side)
    dt = time.perf_counter() - t0
    return side * side / dt / 1e6, "%dx%d region of the sensed image, 12 channels, FP64" % (side, side)


def reduce_over_ranks(dist, torch, ms, matched, device):
    """Whole-job figures of one timed region: the slowest rank's time (max)
    and the points matched by all ranks (sum).  `dist` None = one rank."""
    if dist is None:
        return float(ms), int(matched)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([int(matched)], dtype=torch.int64, device=device)
    dist.all_reduce(n)
    return float(t.item()), int(n.item())


def job_value(matched_all, steps, ms_max):
    """Matched control points per second over the whole job."""
    return matched_all * steps / (ms_max * 1e-3)


def corr_flops(pair, z=12):
    P = (2 * pair.R + 1) ** 2
    return 2.0 * pair.m * pair.m * z * P


def fft_side(pair):
    return next((L for L in FFT_SIZES if pair.m + 2 * pair.R <= L), None)


def fft_flops_mrl(m, R, L, z=12):
    """Work of the Fourier correlation per point, counting 5 L log2 L flop per
    complex length-L transform: per channel m + 2R row and L column
    transforms, 12 flop per cross-spectrum bin of the half spectrum; then
    L/2 + 1 column and 2R + 1 row inverse transforms."""
    t = 5.0 * L * math.log2(L)
    P1 = 2 * R + 1
    return z * ((m + 2 * R + L) * t + 12.0 * L * (L // 2 + 1)) + (L // 2 + 1 + P1) * t


def fft_flops(pair, z=12):
    return fft_flops_mrl(pair.m, pair.R, fft_side(pair), z)


def fp32_peak(pk):
    """FP32 TFLOP/s denominator and its source: the library's own FMA
    microbenchmark (the faster of scalar FFMA and paired FFMA2 chains) when
    it ran, else the nominal figure."""
    if pk.get("fp32"):
        return pk["fp32"], pk["fp32_src"]
    return FP32_PEAK_TFLOPS, "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (nominal: the microbenchmark did not run)"


def form_roofline(form, pair, per_launch_ms, processed, pk, workload, path, option=0):
    """Roofline of a form's correlation kernel (the concrete form `path` the
    steps ran): the algorithmic work of the points it processed over its mean
    launch time (CUDA events), against the peak of the unit that bounds it."""
    per_point = CORR_TRAFFIC_PER_POINT_SAR2048.get((form, path)) if workload == "sar2048" else None
    traffic = per_point * processed if per_point and (pair.m, pair.R) == (81, 20) else None
    secs = per_launch_ms * 1e-3
    peak32, fp32_src = fp32_peak(pk)
    if path == 6:  # the Fourier correlation, on F32 cubes or BF16 cubes widened as read
        L = option or fft_side(pair)
        ach = fft_flops_mrl(pair.m, pair.R, L) * processed / secs / 1e12
        return {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
                "frac": ach / peak32, "traffic": traffic,
                "kernel": "k_corr_fft<%d> (FP32 Fourier correlation, Eq. 13, %s cubes)" % (
                    L, "BF16" if form == "bf16" else "F32"),
                "peak_src": fp32_src,
                "work": "5 L log2 L flop per length-L transform (z (m+2R+L) forward, L/2+1+2R+1 inverse) "
                        "+ 12 flop per cross-spectrum bin, per processed point"}
    ach = corr_flops(pair) * processed / secs / 1e12
    if path in (3, 4, 5):
        return {"bound": "tensor", "achieved": ach, "peak": pk["bf16"], "unit": "TFLOP/s",
                "frac": ach / pk["bf16"], "traffic": traffic,
                "kernel": PATH_NAMES[path] + " (bf16 operands, fp32 accumulate)",
                "peak_src": "bf16_tflops burst, %s" % pk["src"],
                "work": "2*m^2*z*(2R+1)^2 flop per processed point"}
    return {"bound": "alu", "achieved": ach, "peak": peak32, "unit": "TFLOP/s",
            "frac": ach / peak32, "traffic": traffic,
            "kernel": "k_corr_f32 (direct FP32 FMA)", "peak_src": fp32_src,
            "work": "2*m^2*z*(2R+1)^2 flop per processed point"}

# Descriptor variants compared under noise: the paper's SFOC, F-SFOC (first
# order only, Sec. 4.2) and the two weaker smoothings of Fig. 3 (Sec. 2.1).
NOISE_VARIANTS = {
    "SFOC": {},
    "F-SFOC": {"first_order_only": True},
    "SFOC plain Gaussian": {"dil": (1,)},
    "SFOC unsmoothed": {"sigma_d1": 0.0, "sigma_d2": 0.0},
}
# Sec. 4.3: variances 0..0.01 step 0.001 (Gaussian) and 0..0.1 step 0.01 (speckle)
NOISE_LEVELS = {"gaussian": [round(0.001 * i, 3) for i in range(11)],
                "speckle": [round(0.01 * i, 2) for i in range(11)]}
NOISE_TEMPLATE = 80  # the template side of the experiment (Sec. 4.3)


def noise_sweep(args):
    """Noise sensitivity (Sec. 4.3) on the GPU path: the average CMR of each
    descriptor variant over four seeded pairs as noise of growing variance is
    added to the sensed image.  Pairs stand in for the paper's
    optical-to-infrared cases: 1024^2 optical-like reference, sensed image an
    inverting piecewise-linear map of the reference shifted by an integer s in
    [-8, 8]^2; 196 block-gradient points picked on the clean sensed image;
    template 80 x 80 (the paper's), search radius 10.  A match is correct
    within 1.5 px of -s (Sec. 4.1); CMR = correct / matched.  The noise of a
    (pair, kind, level) is drawn once and shared by all variants."""
    import numpy as np
    import torch
    from workloads import add_noise, inverting_pair_512
    import paper_2202_13347_gb300 as pkg
    pkg.build()
    b = pkg.load()
    torch.cuda.set_device(0)
    ctx = b.Context(torch.cuda.current_device())
    # build rate of each variant's cube (CUDA events, median of 10) on the
    # first pair's sensed image: the variants run other smoothing kernels
    # than the paper's configuration
    build_mpix = {}
    probe = inverting_pair_512(seed=4301, H=1024, W=1024, n_side=14, m=NOISE_TEMPLATE, R=10)
    d_probe = torch.from_numpy(probe.sen).cuda()
    for v, kw in NOISE_VARIANTS.items():
        pv = b.params(**kw)
        cube = ctx.sfoc_build(d_probe, p=pv)
        for _ in range(2):
            cube = ctx.sfoc_build(d_probe, p=pv, out=cube)       # rebuilt in place: no allocation timed
        ts = []
        stream = torch.cuda.current_stream()
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cube = ctx.sfoc_build(d_probe, p=pv, out=cube)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        build_mpix[v] = round(probe.sen.size / (statistics.median(ts) * 1e-3) / 1e6, 1)
    seeds = (4301, 4302, 4303, 4304)
    cmr = {v: {k: np.zeros(len(L)) for k, L in NOISE_LEVELS.items()} for v in NOISE_VARIANTS}
    n_points = 0
    t0 = time.perf_counter()
    for seed in seeds:
        pair = inverting_pair_512(seed=seed, H=1024, W=1024, n_side=14, m=NOISE_TEMPLATE, R=10)
        n_points += len(pair.points)
        d_ref = torch.from_numpy(pair.ref).cuda()
        d_pts = torch.from_numpy(pair.points).cuda()
        prm = {v: b.params(**kw) for v, kw in NOISE_VARIANTS.items()}
        ref_cubes = {v: ctx.sfoc_build(d_ref, p=prm[v]) for v in NOISE_VARIANTS}
        for kind, levels in NOISE_LEVELS.items():
            for li, var in enumerate(levels):
                rng = np.random.default_rng([seed, 0 if kind == "gaussian" else 1, li])
                d_sen = torch.from_numpy(add_noise(rng, pair.sen, kind, var)).cuda()
                for v in NOISE_VARIANTS:
                    sen_cube = ctx.sfoc_build(d_sen, p=prm[v])
                    raw = ctx.fastncc_match(ref_cubes[v], sen_cube, d_pts, pair.m, pair.R)["raw"].cpu().numpy()
                    ok = raw[:, 5] == 0
                    off = np.stack([raw[:, 3].view(np.float32), raw[:, 4].view(np.float32)], 1).astype(np.float64)
                    correct = ok & (np.linalg.norm(off - pair.truth, axis=1) <= 1.5)
                    cmr[v][kind][li] += correct.sum() / max(1, int(ok.sum())) / len(seeds)
                    del sen_cube
        del ref_cubes
    line = {"experiment": "noise sensitivity (Sec. 4.3)", "metric": "average CMR", "pairs": len(seeds),
            "points": n_points, "template": NOISE_TEMPLATE, "search_radius": 10, "tolerance_px": 1.5,
            "noise_on": "sensed image", "levels": NOISE_LEVELS,
            "cmr": {v: {k: [round(float(x), 4) for x in a] for k, a in d.items()} for v, d in cmr.items()},
            "sfoc_build_mpix_s": build_mpix, "build_image": "1024x1024",
            "data": "synthetic", "seconds": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------

BATCH_FORMS = ("bf16batch", "f32batch", "f32plain")
PATH_NAMES = {1: "k_corr_f32 (direct FP32)", 3: "k_corr_tc (Toeplitz tcgen05)", 4: "k_corr_tc_col (column tcgen05)",
              5: "k_corr_tc_band (band tcgen05)", 6: "k_corr_fft (FP32 Fourier, Eq. 13)"}


def class_flops(path, cls, m, R, z=12):
    """Algorithmic work per processed point of one correlation class: the
    direct-equivalent 2 m^2 z (2R+1)^2 flop for the direct and tensor-core
    forms, the transform count for the Fourier form (cls = its side)."""
    if path == 6:
        return fft_flops_mrl(m, R, cls, z)
    return 2.0 * m * m * z * (2 * R + 1) ** 2


def corr_option(b, name):
    return {"auto": b.CORR_AUTO, "igemm_tc": b.CORR_IGEMM_TC, "band": b.CORR_TC_BAND, "column": b.CORR_TC_COLUMN,
            "fft": b.CORR_FFT, "direct": b.CORR_DIRECT_F32}[name]


def run_batch_form(b, torch, ctx, pairs, form, steps, warmup, corr_name="auto"):
    p = b.params(dtype=b.DTYPE_BF16 if form == "bf16batch" else b.DTYPE_F32)
    corr = b.CORR_DIRECT_F32 if form == "f32plain" else corr_option(b, corr_name)
    n = len(pairs)
    d_refs = [torch.from_numpy(q.ref).cuda() for q in pairs]
    d_sens = [torch.from_numpy(q.sen).cuda() for q in pairs]
    d_pts = [torch.from_numpy(q.points).cuda() for q in pairs]
    outs = [torch.empty((len(q.points), 6), dtype=torch.int32, device="cuda") for q in pairs]
    ms_, Rs_ = [q.m for q in pairs], [q.R for q in pairs]
    if form == "f32plain":
        # pairs one after the other; each pair's cubes are rebuilt in place
        cr, cs = [None] * n, [None] * n

        def step():
            for i in range(n):
                cr[i] = ctx.sfoc_build(d_refs[i], p=p, out=cr[i])
                cs[i] = ctx.sfoc_build(d_sens[i], p=p, out=cs[i])
                outs[i].copy_(ctx.fastncc_match(cr[i], cs[i], d_pts[i], ms_[i], Rs_[i], corr_path=corr)["raw"])
    else:
        def step():
            ctx.register_batch(d_refs, d_sens, d_pts, ms_, Rs_, p=p, corr_path=corr, outs=outs)
    t0 = time.perf_counter()
    step()  # the first call: plan, autotuner measurements, graph capture
    ctx.sync()
    prep_s = time.perf_counter() - t0
    for _ in range(warmup):
        step()
    ctx.sync()
    stream = torch.cuda.current_stream()
    l0 = ctx.launch_count
    evs = []
    torch.cuda.synchronize()
    t_start = time.monotonic()
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    t_end = time.monotonic()
    launches = ctx.launch_count - l0
    ctx.sync()
    ms = [a.elapsed_time(c) for a, c in evs]
    status = [o[:, 5].cpu() for o in outs]
    matched = int(sum(int((st == 0).sum()) for st in status))
    processed = [int(((st == 0) | (st == 3)).sum()) for st in status]
    # stage breakdown: one more step with per-stage events (a plan runs stage
    # by stage while they are on)
    info = ctx.plan_info() if form != "f32plain" else None
    ctx.enable_timing(True)
    ctx.reset_timing()
    step()
    stages = ctx.stage_times()
    scopes = ctx.stage_scopes("correlation")
    ctx.enable_timing(False)
    tune = {}
    if corr in (b.CORR_AUTO, b.CORR_IGEMM_TC):
        for q in pairs:
            e = ctx.autotune_entry(p.cube_dtype, q.m, q.R, 0 if corr == b.CORR_AUTO else 1)
            if e:
                tune["%d,%d" % (q.m, q.R)] = {"path": e["path"], "option": e["option"],
                                              "candidates_ms": {"%d/%d" % (c[0], c[1]): round(c[2], 4)
                                                                for c in e["candidates"]}}
    return dict(ms=sum(ms), ms_steps=ms, matched=matched, processed=processed, stages=stages, scopes=scopes,
                info=info, launches=launches, p=p, corr=corr, outs=outs, prep_s=prep_s, tune=tune,
                t_timed=(t_start, t_end))


# DRAM bytes per processed point of a band-form class, by (template side,
# band instance NQ), from ncu captures of the kernel as it stands, each of the
# 2048x2048 pair's 1000 points matched with forced band form at one (m, R):
# m = 101, R = 40 (851 processed; 745.06 MB read + 44.46 MB written per
# launch) and m = 81, R = 36 (879 points in bounds; 359.81 MB + 30.00 MB).  A
# batched class of the same template side and instance gets this times its
# processed points (its radii range over R 33-40).
BAND_TRAFFIC_PER_POINT = {(101, 6): (745.062144e6 + 44.461312e6) / 851,
                          (81, 6): (359.80928e6 + 29.997056e6) / 879}


def batch_roofline(form, pairs, r, pk):
    """Roofline of the dominant correlation kernel of a batched form: per
    class (one persistent launch), the algorithmic work of the points it
    processed over its launch time (CUDA events of the stage-by-stage run),
    against the peak of the unit that bounds it; the class with the longest
    launch is reported, all classes beside it."""
    peak32, src32 = fp32_peak(pk)
    rows = []
    if r["info"] is None:  # pairs in order: every launch is the direct kernel
        fl = sum(class_flops(1, 0, q.m, q.R) * r["processed"][i] for i, q in enumerate(pairs))
        secs = sum(r["scopes"]) * 1e-3
        rows.append(dict(kernel=PATH_NAMES[1], path=1, cls=0, launches=len(r["scopes"]), ms=sum(r["scopes"]),
                         flops=fl, items=sum(r["processed"])))
    else:
        k = 0
        for c in r["info"]["classes"]:
            nl = c["launches"]
            ms = sum(r["scopes"][k:k + nl])
            k += nl
            fl = sum(class_flops(c["path"], c["cls"], pairs[i].m, pairs[i].R) * r["processed"][i] for i in c["pairs"])
            tm = sorted({pairs[i].m for i in c["pairs"]})
            tr = sorted({pairs[i].R for i in c["pairs"]})
            per_pt = BAND_TRAFFIC_PER_POINT.get((tm[0], c["cls"])) if c["path"] == 5 and len(tm) == 1 else None
            npts = sum(r["processed"][i] for i in c["pairs"])
            rows.append(dict(kernel=PATH_NAMES.get(c["path"], str(c["path"])), path=c["path"], cls=c["cls"],
                             launches=nl, ms=ms, flops=fl, items=c["items"], m=tm, R=[tr[0], tr[-1]],
                             traffic=per_pt * npts / nl if per_pt else None))
    out = []
    for row in rows:
        tc = row["path"] in (3, 4, 5)
        peak = pk["bf16_sus"] if tc else peak32
        # work per launch over mean launch time = the class's work over its launches' summed time
        ach = row["flops"] / (row["ms"] * 1e-3) / 1e12 if row["ms"] > 0 else 0.0
        out.append(dict(row, achieved=ach, peak=peak, frac=ach / peak, bound="tensor" if tc else "alu"))
    top = max(out, key=lambda x: x["ms"])
    tc = top["path"] in (3, 4, 5)
    return {"bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"], "unit": "TFLOP/s",
            "frac": top["frac"], "traffic": top.get("traffic"), "kernel": top["kernel"] + " class %d" % top["cls"],
            "launch_ms": top["ms"] / max(1, top["launches"]),
            "peak_src": ("bf16_tflops_sustained (%s): timed inside a long step" % pk["src"]) if tc else src32,
            "work": ("2*m^2*z*(2R+1)^2 flop per processed point" if top["path"] != 6 else
                     "5 L log2 L flop per transform + 12 flop per cross-spectrum bin, per processed point"),
            "classes": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in x.items() if k != "flops"}
                        for x in out]}


def batch_e2e(b, torch, ctx, pairs, p, corr, steps):
    """The same step through the C ABI from host buffers (pinned): each
    step's images and point sets are copied in and its results copied out
    inside the timed region.  The steps are a stream of submissions
    (fastncc_submit_batch_host): step k + 1 is submitted before step k's
    results are waited for (fastncc_wait_batch_host), so its copies run
    while step k is matched; the region ends when the last step's results
    are on the host.  Alternate steps write alternate result buffers.  The
    synchronous call (fastncc_register_batch_host, one step per call) is
    timed afterwards as a side figure."""
    h_refs = [torch.from_numpy(q.ref).pin_memory() for q in pairs]
    h_sens = [torch.from_numpy(q.sen).pin_memory() for q in pairs]
    h_pts = [torch.from_numpy(q.points).pin_memory() for q in pairs]
    outs = [[torch.empty((len(q.points), 6), dtype=torch.int32).pin_memory() for q in pairs] for _ in range(2)]
    ms_, Rs_ = [q.m for q in pairs], [q.R for q in pairs]
    for _ in range(2):  # plan and graph of the staged buffers
        ctx.register_batch_host(h_refs, h_sens, h_pts, ms_, Rs_, p=p, corr_path=corr, outs=outs[0])
    built0 = ctx.plan_info().get("plans_built")
    # Python's cyclic garbage collector stays off while the calls are timed (as
    # timeit does): a full collection over the benchmark's own objects is not
    # part of the library call
    import gc
    gc.collect()
    gc.disable()
    done = []
    try:
        tickets = []
        t0 = time.perf_counter()
        for k in range(steps):
            t, _ = ctx.submit_batch_host(h_refs, h_sens, h_pts, ms_, Rs_, p=p, corr_path=corr, outs=outs[k % 2])
            tickets.append(t)
            if k >= 1:
                ctx.wait_batch_host(tickets[k - 1])
                done.append(time.perf_counter())
        ctx.wait_batch_host(tickets[-1])
        done.append(time.perf_counter())
        total = done[-1] - t0
        sync_t = []
        for _ in range(steps):
            s0 = time.perf_counter()
            ctx.register_batch_host(h_refs, h_sens, h_pts, ms_, Rs_, p=p, corr_path=corr, outs=outs[0])
            sync_t.append(time.perf_counter() - s0)
    finally:
        gc.enable()
    built1 = ctx.plan_info().get("plans_built")
    last = outs[(steps - 1) % 2]
    matched = sum(int((o[:, 5] == 0).sum()) for o in last)
    same = all(torch.equal(x, y) for x, y in zip(outs[0], outs[1])) if steps >= 2 else None
    h2d = sum(x.numel() * 4 for x in h_refs + h_sens + h_pts)
    d2h = sum(o.numel() * 4 for o in last)
    # the copy rate these host buffers get on their own (outside the timed calls)
    gbs = None
    try:
        dev = [torch.empty_like(x, device="cuda") for x in h_refs + h_sens]
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        for d, x in zip(dev, h_refs + h_sens):
            d.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        gbs = round(sum(x.numel() * 4 for x in h_refs + h_sens) / (time.perf_counter() - c0) / 1e9, 1)
        del dev
    except RuntimeError:  # a side figure: no device copy, no rate
        pass
    return dict(ms=1e3 * total, steps=steps, matched=matched, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                step_done_ms=[round(1e3 * (done[i] - (done[i - 1] if i else t0)), 1) for i in range(len(done))],
                sync_call_ms=[round(1e3 * x, 1) for x in sync_t], results_equal_across_steps=same,
                h2d_gbs_alone=gbs,
                plans_built_in_timed_calls=(built1 - built0) if built0 is not None and built1 is not None else None)


def batch_oracle_sample(pairs, seed, n_pairs=16, per_pair=2):
    """A seeded sample of (pair, point) indices of the batch."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(pairs), min(n_pairs, len(pairs)), replace=False))
    out = []
    for i in sel:
        k = min(per_pair, len(pairs[i].points))
        out.append((int(i), np.sort(rng.choice(len(pairs[i].points), k, replace=False))))
    return out


def batch_cpu_baseline(pairs, outs, seed=99):
    """The oracle as it stands on a seeded sample of the batch's points (2 in
    each of 16 pairs: about 15 s on 16 host cores), and the agreement of the
    GPU results on those points with it: offsets equal, near-ties (oracle
    best-vs-second margin <= 2e-4) and NCC error against the FP64 oracle."""
    import numpy as np
    import oracle
    oracle.build()
    sample = batch_oracle_sample(pairs, seed)
    matched, dt = 0, 0.0
    eq = ties = valid = 0
    err = 0.0
    for i, idx in sample:
        q = pairs[i]
        t0 = time.perf_counter()
        o = oracle.match_pair(q.ref, q.sen, q.points[idx], q.m, q.R)
        dt += time.perf_counter() - t0
        matched += int((o["status"] == 0).sum())
        g = outs[i][torch_index(idx)].cpu().numpy()
        ok = np.isin(o["status"], [0, 3])
        valid += int(ok.sum())
        same = ok & (g[:, 0] == o["dx"]) & (g[:, 1] == o["dy"])
        eq += int(same.sum())
        ties += int((ok & (o["margin"] <= 2e-4)).sum())
        if same.any():
            gn = g[:, 2].view(np.float32).astype(np.float64)
            err = max(err, float(np.abs(gn[same] - o["ncc"][same]).max()))
    n = sum(len(idx) for _, idx in sample)
    mpix, region = oracle_sfoc_mpix(pairs[0])
    cpu = dict(value=matched / dt, unit=UNIT, cores=oracle.num_threads(), kind="oracle",
               sample="%d points (2 in each of %d seeded pairs) of %d, FP64 SFOC on their windows only, Eq. 8 NCC"
               % (n, len(sample), sum(len(q.points) for q in pairs)),
               seconds=dt, sfoc_mpix_s=mpix, sfoc_sample=region)
    parity = dict(points=n, valid=valid, offsets_equal=eq, near_ties=ties, ncc_err_max_vs_fp64=err,
                  note="GPU result of the line's form against the unrounded FP64 oracle on the sampled points")
    return cpu, parity


def torch_index(idx):
    import torch
    return torch.from_numpy(idx)


def reference_batch(args, rank):
    """The reference arm on the batched workload: the oracle as it stands on
    the host cores, each step a bounded seeded sample (4 points) of the same
    64-pair batch; rank 0 only."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    pairs, desc = batch_workload(0, min(16, os.cpu_count() or 1), args.pairs, args.scale)
    steps_t, matched, n_sample = [], 0, 4
    for i in range(args.warmup + args.steps):
        sample = batch_oracle_sample(pairs, 1000 + i, n_pairs=n_sample, per_pair=1)
        t0 = time.perf_counter()
        ok = 0
        for pi, idx in sample:
            q = pairs[pi]
            o = oracle.match_pair(q.ref, q.sen, q.points[idx], q.m, q.R)
            ok += int((o["status"] == 0).sum())
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            steps_t.append(dt)
            matched += ok
    tot = sum(steps_t)
    value = matched / tot
    mpix, region = oracle_sfoc_mpix(pairs[0])
    sample = "%d seeded points per step (1 in each of %d seeded pairs) of %d, FP64 SFOC on their windows, Eq. 8 NCC" % (
        n_sample, n_sample, sum(len(q.points) for q in pairs))
    config = {"workload": desc, "pairs_per_rank": len(pairs), "points_per_rank": sum(len(q.points) for q in pairs),
              "z": 12, "form": "bf16batch"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample, "sfoc_mpix_s": mpix, "sfoc_sample": region},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main_batch(args, torch, dist, rank, world, gpu_index):
    import paper_2202_13347_gb300 as pkg
    pkg.build()
    b = pkg.load()
    strong = args.scaling == "strong" and world > 1
    pairs, desc = batch_workload(0 if strong else rank, min(16, os.cpu_count() or 1), args.pairs, args.scale)
    mine = list(range(len(pairs)))
    if strong:  # one job, its pairs balanced over the ranks
        from paper_2202_13347_gb300 import shard
        job = pairs
        costs = [shard.pair_cost(len(q.points), q.m, q.R, q.ref.size + q.sen.size) for q in job]
        mine = shard.shard_pairs(costs, world)[rank]
        pairs = [job[i] for i in mine]
        desc += "; pairs of one job balanced over %d ranks by cost" % world
    px = sum(q.ref.size + q.sen.size for q in pairs)
    n_points = sum(len(q.points) for q in pairs)
    config = {"workload": desc, "pairs_per_rank": len(pairs), "points_per_rank": n_points, "pixels_per_rank": px,
              "z": 12, "l2": "not flushed: every step reads %.1f GB of images and cubes, far above the 129 MB L2"
              % (px * 4 / 1e9 * 18)}
    ctx = b.Context(torch.cuda.current_device())
    forms = [f for f in (args.forms or ",".join(BATCH_FORMS)).split(",") if f]
    pk = peaks()
    try:
        mp = ctx.measure_peaks()
        pk.update(fp32=max(mp["fp32_tflops"], mp["fp32x2_tflops"]), fp32_scalar=mp["fp32_tflops"],
                  fp32_src="measured by sfoc_measure_peaks: %s FMA chains (scalar %.1f, paired %.1f TFLOP/s)" % (
                      "paired FFMA2" if mp["fp32x2_tflops"] > mp["fp32_tflops"] else "scalar FFMA",
                      mp["fp32_tflops"], mp["fp32x2_tflops"]), microbench=mp)
    except Exception as e:  # noqa: BLE001
        pk.update(microbench={"error": str(e)})
    results = {}
    for form in forms:
        try:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            steps = args.steps if form != "f32plain" else max(3, min(args.steps, 5))
            with ClockSampler(gpu_index) as cs:
                r = run_batch_form(b, torch, ctx, pairs, form, steps, args.warmup if form != "f32plain" else 1,
                                   args.corr)
                cs.mark(*r["t_timed"])
            r["steps"] = steps
            r["ms_max"], r["matched_all"] = reduce_over_ranks(dist, torch, r["ms"], r["matched"], "cuda")
            r["clocks"] = cs.summary()
            results[form] = r
            # the headline form's end-to-end calls right after its own steps, before
            # the FP32 forms: after those (hundreds of cube allocations and seconds of
            # FP32 work) the host copies of alternate calls were seen to run at a
            # tenth of their rate, with no kernel running beside them
            if form == "bf16batch" and not args.no_e2e:
                r["e2e_raw"] = batch_e2e(b, torch, ctx, pairs, r["p"], r["corr"], max(3, args.steps))
        except b.SfocError as e:
            results[form] = {"error": str(e)}
        if form != forms[-1] and form != "bf16batch":
            ctx.release_plans()  # the next form builds its own cubes
    ok = [f for f in forms if "error" not in results.get(f, {"error": 1})]
    if not ok:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": {f: results[f].get("error") for f in forms}}))
        sys.exit(1)

    def summarize(r, form):
        per_step = {k: v[0] for k, v in r["stages"].items()}  # the one stage-by-stage step
        sfoc_ms = per_step["steer"] + per_step["smooth"]
        return dict(value=job_value(r["matched_all"], r["steps"], r["ms_max"]), ms_per_step=r["ms_max"] / r["steps"],
                    steps=r["steps"], sfoc_mpix_s=px / (sfoc_ms * 1e-3) / 1e6 if sfoc_ms > 0 else None,
                    stage_ms_per_step={k: round(v, 3) for k, v in per_step.items()},
                    roofline=batch_roofline(form, pairs, r, pk), matched_per_step=r["matched"],
                    gpu_launches=r["launches"], launches_per_step=r["launches"] / r["steps"], clocks=r["clocks"],
                    first_call_s=round(r["prep_s"], 2), graph=bool(r["info"] and r["info"].get("graph")),
                    autotune=r["tune"] or None)

    summ = {f: summarize(results[f], f) for f in ok}
    main_form = "bf16batch" if "bf16batch" in summ else max(summ, key=lambda f: summ[f]["value"])
    main = summ[main_form]
    r0 = results[main_form]
    e2e = None
    if not args.no_e2e and main_form != "f32plain":
        er = r0.get("e2e_raw") or batch_e2e(b, torch, ctx, pairs, r0["p"], r0["corr"], max(3, args.steps))
        if dist:
            dist.barrier()
        ms_max, matched_all = reduce_over_ranks(dist, torch, er["ms"], er["matched"] * er["steps"], "cuda")
        e2e = dict(value=matched_all / (ms_max * 1e-3), unit=UNIT, h2d_bytes_per_step=er["h2d_bytes_per_step"],
                   d2h_bytes_per_step=er["d2h_bytes_per_step"], ms_per_step=ms_max / er["steps"],
                   call="fastncc_submit_batch_host + fastncc_wait_batch_host (pinned host buffers; step k+1 "
                        "submitted before step k is waited for)",
                   step_done_ms=er["step_done_ms"], results_equal_across_steps=er["results_equal_across_steps"],
                   sync_call="fastncc_register_batch_host", sync_call_ms=er["sync_call_ms"],
                   h2d_gbs_alone=er["h2d_gbs_alone"], plans_built_in_timed_calls=er["plans_built_in_timed_calls"])
    gathered = None
    if strong:  # the final collective: every rank's results to rank 0, in the job's order
        import numpy as np
        from paper_2202_13347_gb300 import shard
        offs = np.cumsum([0] + [len(q.points) for q in job])
        idx = np.concatenate([np.arange(offs[i], offs[i + 1]) for i in mine]) if mine else np.zeros(0, np.int64)
        rows = (np.concatenate([o.cpu().numpy() for o in r0["outs"]]) if mine else np.zeros((0, 6), np.int32))
        full = shard.gather_results(dist, rank, world, int(offs[-1]), idx, rows)
        if rank == 0:
            gathered = {"points": int(full.shape[0]), "matched": int((full[:, 5] == 0).sum())}
    cpu, parity = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu, parity = batch_cpu_baseline(pairs, r0["outs"])
        except Exception as e:  # noqa: BLE001
            cpu = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": main["steps"],
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "strong" if strong else "weak", "vs_baseline": None,
            "dtype": "bf16" if main_form == "bf16batch" else "f32",
            "data": "synthetic", "config": dict(config, form=main_form), "roofline": main["roofline"],
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": main["gpu_launches"], "clocks": main["clocks"],
            "sfoc_mpix_s": main["sfoc_mpix_s"], "stage_ms_per_step": main["stage_ms_per_step"], "parity": parity,
            "gathered": gathered,
            "forms": {f: {k: v for k, v in sm.items() if k not in ("clocks",)} for f, sm in summ.items()},
            "bf16batch_over_f32plain": (summ["bf16batch"]["value"] / summ["f32plain"]["value"]
                                        if "bf16batch" in summ and "f32plain" in summ else None),
            "peaks": {"hbm_gbs": pk["hbm"], "bf16_tflops": pk["bf16"], "bf16_tflops_sustained": pk["bf16_sus"],
                      "src": pk["src"] + " (MEASURED_PEAKS.json)", "microbench": pk.get("microbench")},
            "errors": {f: results[f]["error"] for f in forms if "error" in results[f]} or None}
    print(json.dumps(line))


def main():
    args = parse()
    if args.noise_sweep:
        return noise_sweep(args)
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        if torch.cuda.is_available():
            torch.cuda.set_device(0)

    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if os.environ.get(
        "CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    if args.workload == "mixed64":
        if args.impl == "reference":
            return reference_batch(args, rank)
        return main_batch(args, torch, dist, rank, world, gpu_index)
    pair, desc = workload(args.workload, rank)
    if args.template > 0 or args.radius >= 0:
        pair.m = args.template if args.template > 0 else pair.m
        pair.R = args.radius if args.radius >= 0 else pair.R
        desc = "%s, with m=%d, R=%d instead" % (desc, pair.m, pair.R)
    config = {"workload": desc, "H": int(pair.ref.shape[0]), "W": int(pair.ref.shape[1]),
              "points_per_pair": int(len(pair.points)), "m": pair.m, "R": pair.R, "z": 12,
              "pairs_per_rank": 1, "l2": "flushed between timed steps (256 MB write)"}

    if args.impl == "reference":
        # the CPU oracle as it stands, on a bounded sample of the same workload
        if rank != 0:
            return
        import oracle
        oracle.build()
        steps_t = []
        matched = 0
        n_sample = 8
        for i in range(args.warmup + args.steps):
            import numpy as np
            rng = np.random.default_rng(1000 + i)
            idx = np.sort(rng.choice(len(pair.points), n_sample, replace=False))
            t0 = time.perf_counter()
            o = oracle.match_pair(pair.ref, pair.sen, pair.points[idx], pair.m, pair.R)
            dt = time.perf_counter() - t0
            if i >= args.warmup:
                steps_t.append(dt)
                matched += int((o["status"] == 0).sum())
        tot = sum(steps_t)
        value = matched / tot
        mpix, region = oracle_sfoc_mpix(pair)
        sample = "%d seeded points of %d per step, FP64 SFOC on their windows, Eq. 8 NCC" % (n_sample, len(pair.points))
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
                "impl": "reference",
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": sample, "sfoc_mpix_s": mpix, "sfoc_sample": region},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import paper_2202_13347_gb300 as pkg
    pkg.build()
    b = pkg.load()
    ctx = b.Context(torch.cuda.current_device())
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    forms = [f for f in (args.forms or "bf16,f32,f32direct").split(",") if f]
    pk = peaks()
    try:  # the FP32 peak of this device, by the library's own microbenchmark
        mp = ctx.measure_peaks()
        pk.update(fp32=max(mp["fp32_tflops"], mp["fp32x2_tflops"]), fp32_scalar=mp["fp32_tflops"],
                  fp32_src="measured by sfoc_measure_peaks: %s FMA chains (scalar %.1f, paired %.1f TFLOP/s)" % (
                      "paired FFMA2" if mp["fp32x2_tflops"] > mp["fp32_tflops"] else "scalar FFMA",
                      mp["fp32_tflops"], mp["fp32x2_tflops"]), microbench=mp)
    except Exception as e:  # noqa: BLE001
        pk.update(microbench={"error": str(e)})
    results = {}
    clocks = None
    for form in forms:
        try:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            with ClockSampler(gpu_index) as cs:
                r = run_form(b, torch, ctx, pair, form, args.steps, args.warmup, flush, args.corr)
                cs.mark(*r["t_timed"])
            r["ms_max"], r["matched_all"] = reduce_over_ranks(dist, torch, r["ms"], r["matched"], "cuda")
            r["clocks"] = cs.summary()
            results[form] = r
        except b.SfocError as e:
            results[form] = {"error": str(e)}
    main_form = next((f for f in forms if "error" not in results.get(f, {"error": 1})), None)
    if main_form is None:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "error": {f: results[f].get("error") for f in forms}}))
        sys.exit(1)

    def summarize(r, form):
        st = r["stages"]
        per_step = {k: v[0] / args.steps for k, v in st.items()}
        sfoc_ms = per_step["steer"] + per_step["smooth"]
        corr_ms, corr_n = st["correlation"]
        per_launch = corr_ms / max(1, corr_n)
        roof = form_roofline(form, pair, per_launch, r["valid"], pk, args.workload, r["path"], r["option"])
        return dict(value=job_value(r["matched_all"], args.steps, r["ms_max"]), ms_per_step=r["ms_max"] / args.steps,
                    sfoc_mpix_s=2 * pair.ref.size / (sfoc_ms * 1e-3) / 1e6 if sfoc_ms > 0 else None,
                    stage_ms_per_step={k: round(v, 4) for k, v in per_step.items()}, roofline=roof,
                    matched_per_step=r["matched"], gpu_launches=r["launches"], clocks=r["clocks"])

    summ = {f: summarize(results[f], f) for f in forms if "error" not in results[f]}
    main_form = max(summ, key=lambda f: summ[f]["value"])  # the fastest form heads the line
    main = summ[main_form]
    r0 = results[main_form]
    e2e = None
    if not args.no_e2e:
        r = run_e2e(b, torch, ctx, pair, r0["p"], r0["corr"], max(3, args.steps))
        if dist:
            dist.barrier()
        ms_max, matched_all = reduce_over_ranks(dist, torch, r["ms"], r["matched"] * r["steps"], "cuda")
        e2e = dict(value=matched_all / (ms_max * 1e-3), unit=UNIT, h2d_bytes_per_step=r["h2d_bytes_per_step"],
                   d2h_bytes_per_step=r["d2h_bytes_per_step"], ms_per_step=ms_max / r["steps"])
    # the rows around matching and the CPU baseline run on rank 0 only; a
    # failure in one of them is reported in its own entry, not in place of
    # the line
    def aux(fn, *a):
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001
            return {"error": "%s: %s" % (type(e).__name__, e)}

    ransac, quality, fast, cpu = None, None, None, None
    if rank == 0:
        rq = aux(run_ransac, b, torch, ctx, pair, r0)
        ransac, quality = (rq, None) if isinstance(rq, dict) else rq
        fast = aux(run_fast, torch, ctx, pair, pk["hbm"], 10, 32, 0.05, pk)
        if world == 1 and not args.no_cpu_baseline:
            cb = aux(cpu_baseline, pair)
            if isinstance(cb, tuple):
                cpu, (idx, o) = cb
                for f in summ:
                    summ[f]["parity"] = aux(form_parity, results[f]["raw"], idx, o)
            else:
                cpu = cb
    if rank != 0:
        return
    line = {"metric": METRIC, "value": main["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if main_form == "bf16" else "f32",
            "data": "synthetic", "config": dict(config, form=main_form), "roofline": main["roofline"],
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": main["gpu_launches"], "clocks": main["clocks"],
            "sfoc_mpix_s": main["sfoc_mpix_s"], "stage_ms_per_step": main["stage_ms_per_step"],
            "parity": main.get("parity"),
            "forms": {f: {k: v for k, v in s.items() if k not in ("clocks",)} for f, s in summ.items()},
            "ransac": ransac, "match_quality": quality, "fast": fast, "peaks": {
                "hbm_gbs": pk["hbm"], "bf16_tflops": pk["bf16"], "src": pk["src"] + " (MEASURED_PEAKS.json)",
                "microbench": pk.get("microbench")},
            "errors": {f: results[f]["error"] for f in forms if "error" in results[f]} or None}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
