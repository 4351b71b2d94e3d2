"""The oracle's pins catch plausible mistakes in the oracle.

Each case copies the oracle's C sources, plants one mistake of the kind
the pins exist to catch (a dropped term, a flipped sign, a swapped index, a
transposed operand, a wrong constant of a reading), builds that copy into a
library of its own and runs the oracle pin tests against it in a separate
process: they must fail.  The in-tree oracle is not touched.

Two mutations are not listed because no observable result depends on
them: the Hartley scale of RANSAC's normalisation (any similarity gives
the same model in exact arithmetic; sqrt(2) only conditions the solve) and
an inclusive versus exclusive inlier threshold (they differ only for an
error exactly equal to the threshold).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRCS = ("sfoc_oracle.c", "ransac_oracle.c", "fast_oracle.c")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_fast.py", "tests/test_oracle_ransac.py",
        "tests/test_oracle_rectify.py"]

S, R, F = SRCS
MUTATIONS = [
    ("eq6_cos_sin_swapped", S, "double v = ct[k] * Ix[s] + st[k] * Iy[s];", "double v = st[k] * Ix[s] + ct[k] * Iy[s];"),
    ("eq7_cross_sign", S, "- 2.0 * st[k] * ct[k] * Ixy;", "+ 2.0 * st[k] * ct[k] * Ixy;"),
    ("eq7_cross_factor", S, "- 2.0 * st[k] * ct[k] * Ixy;", "- 1.0 * st[k] * ct[k] * Ixy;"),
    ("scale_sum_dropped", S, "f += p->rectify ? fabs(v) : v;", "f = p->rectify ? fabs(v) : v;"),
    ("norm_without_sqrt", S, "double den = sqrt(n2s) + p->eps;", "double den = n2s + p->eps;"),
    ("unsmoothed_offset", S, "D[c] = Fc[(size_t)(y - ey0) * ew + (x - ex0)];",
     "D[c] = Fc[(size_t)(y - ey0) * ew + (x - ex0) + (x + 1 < W ? 1 : 0)];"),
    ("eq2_sign", S, "gx[(y + K) * n + (x + K)] = -(double)x / (2.0 * OR_PI * s4) * e;",
     "gx[(y + K) * n + (x + K)] = (double)x / (2.0 * OR_PI * s4) * e;"),
    ("dilated_variance", S, "g[t + Kd] = exp(-(double)t * t / (2.0 * sigma_d * sigma_d));",
     "g[t + Kd] = exp(-(double)t * t / (sigma_d * sigma_d));"),
    ("template_transposed", S, "double dt = cube_at(sen, c, ty0 + i, tx0 + j) - tbar;",
     "double dt = cube_at(sen, c, ty0 + j, tx0 + i) - tbar;"),
    ("window_dx_dy_swapped", S, "double ds = cube_at(ref, c, ty0 + i + dy, tx0 + j + dx) - sbar;",
     "double ds = cube_at(ref, c, ty0 + i + dx, tx0 + j + dy) - sbar;"),
    ("flat_threshold", S, "if (vT <= 1e-6 * N) { o->status = OR_FLAT_TEMPLATE; continue; }",
     "if (vT <= 1e-3 * N) { o->status = OR_FLAT_TEMPLATE; continue; }"),
    ("argmax_ties_last", S, "if (best < 0 || v > bv) { best = i; bv = v; }",
     "if (best < 0 || v >= bv) { best = i; bv = v; }"),
    ("parabola_sign", S, "double d = (cm - cp) / (2.0 * den);", "double d = (cp - cm) / (2.0 * den);"),
    ("parabola_clamp", S, "if (d > 0.5) d = 0.5;", "if (d > 0.4) d = 0.4;"),
    ("integral_row_sum", S, "            s += g[(size_t)(y - 1) * W + (x - 1)];",
     "            s = g[(size_t)(y - 1) * W + (x - 1)];"),
    ("eq16_corner_sign", S, "- P[(size_t)y1 * W1 + x0] + P[(size_t)y0 * W1 + x0];",
     "- P[(size_t)y1 * W1 + x0] - P[(size_t)y0 * W1 + x0];"),
    ("ransac_ties_later", R, "        if (sc > bs) {", "        if (sc >= bs) {"),
    ("bilinear_transposed", R,
     "v = (float)((1.0 - ft) * ((1.0 - fu) * p00 + fu * p01) + ft * ((1.0 - fu) * p10 + fu * p11));",
     "v = (float)((1.0 - fu) * ((1.0 - ft) * p00 + ft * p01) + fu * ((1.0 - ft) * p10 + ft * p11));"),
    ("fast_arcs_of_8", F, "for (int j = 1; j < 9; ++j) {", "for (int j = 1; j < 8; ++j) {"),
    ("fast_min_polarity", F, "const float m = mb > md ? mb : md;", "const float m = mb < md ? mb : md;"),
    ("nms_tie_rule", F, "if (before ? !(v > u) : !(v >= u)) return 0;", "if (!(v >= u)) return 0;"),
    ("g2_zero_mean_dropped", S, "        for (int x = 0; x < n; ++x) gxx[y * n + x] -= m;",
     "        for (int x = 0; x < n; ++x) gxx[y * n + x] -= 0.0 * m;"),
    ("gxy_sign", S, "gxy[(y + K) * n + (x + K)] = ((double)x * y / (2.0 * OR_PI * s6)) * e;",
     "gxy[(y + K) * n + (x + K)] = (-(double)x * y / (2.0 * OR_PI * s6)) * e;"),
    ("dilation_rows_undilated", S, "w[(r * u + r * Kd) * n + (r * t + r * Kd)] = g[u + Kd] * g[t + Kd];",
     "w[(u + r * Kd) * n + (r * t + r * Kd)] = g[u + Kd] * g[t + Kd];"),
    ("group_boundary", S, "int g = c < no ? 0 : 1;", "int g = c <= no ? 0 : 1;"),
    ("window_mean_n_minus_1", S, "double sbar = ssum / N;", "double sbar = ssum / (N - 1.0);"),
    ("ncc_without_sqrt", S, "else v = num / sqrt(vS * vT);", "else v = num / (vS * vT);"),
    ("even_template_half", S, "int oracle_template_half(int m) { return (m % 2) ? (m - 1) / 2 : m / 2; }",
     "int oracle_template_half(int m) { return (m % 2) ? (m - 1) / 2 : m / 2 - 1; }"),
    ("refit_second_row_dropped", R, "M[a * nu + c] += r1[a] * r1[c] + r2[a] * r2[c];",
     "M[a * nu + c] += r1[a] * r1[c];"),
    ("rmse_without_sqrt", R, "*rmse = ncm ? sqrt(se / ncm) : 0.0;", "*rmse = ncm ? se / ncm : 0.0;"),
    ("rectify_right_edge_open", R, "if (u >= 0.0 && t >= 0.0 && u <= W - 1 && t <= H - 1) {",
     "if (u >= 0.0 && t >= 0.0 && u < W - 1 && t < H - 1) {"),
    ("rectify_forward_map", R, "for (int k = 0; k < 9; ++k) inv[k] /= inv[8];",
     "for (int k = 0; k < 9; ++k) inv[k] = (k == 0 ? a : k == 1 ? b : k == 2 ? c : k == 3 ? d : k == 4 ? e : "
     "k == 5 ? f : k == 6 ? g : k == 7 ? h : i) / i;"),
    ("angles_over_2pi", S, "        ct[k] = cos(k * OR_PI / no);\n        st[k] = sin(k * OR_PI / no);",
     "        ct[k] = cos(2.0 * k * OR_PI / no);\n        st[k] = sin(2.0 * k * OR_PI / no);"),
    ("radius_floor", S, "return (int)ceil(mult * sigma - 1e-9);", "return (int)floor(mult * sigma + 1e-9);"),
    ("zero_padded_borders", S,
     "for (int qx = -K; qx <= K; ++qx) acc += kr[qx + K] * (double)row[clampi(x - qx, 0, W - 1)];",
     "for (int qx = -K; qx <= K; ++qx) acc += (x - qx < 0 || x - qx >= W) ? 0.0 : "
     "kr[qx + K] * (double)row[clampi(x - qx, 0, W - 1)];"),
    ("eq13_conjugate_on_s", S, "acci[q] += si[q] * tr[q] - sr[q] * ti[q];", "acci[q] += sr[q] * ti[q] - si[q] * tr[q];"),
    ("fast_circle_offset", F, "{1, 3},\n", "{1, 2},\n"),
    ("fast_blocks_rows_by_w", F, "const int y0 = (int)((long long)by * H / grid_y), y1 = (int)((long long)(by + 1) * H / grid_y);",
     "const int y0 = (int)((long long)by * W / grid_y), y1 = (int)((long long)(by + 1) * W / grid_y);"),
    ("rectify_u_from_y", R, "const double u = (inv[0] * x + inv[1] * y + inv[2]) / w;",
     "const double u = (inv[1] * x + inv[0] * y + inv[2]) / w;"),
    ("norm_over_all_channels", S, "for (int k = 0; k < no; ++k) n2s += D[g * no + k] * D[g * no + k];",
     "for (int k = 0; k < z; ++k) n2s += D[k] * D[k];"),
    ("eps_inside_sqrt", S, "double den = sqrt(n2s) + p->eps;", "double den = sqrt(n2s + p->eps);"),
    ("rates_averaged", S, "                D[c] = acc;", "                D[c] = acc / p->n_dil;"),
    ("ransac_projective_sign", R, "        r1[6] = -x * xp; r1[7] = -y * xp;", "        r1[6] = x * xp; r1[7] = -y * xp;"),
    ("eq9_square_plane", S, "g2[i] += v * v;", "g2[i] += v;"),
    ("fast_threshold_inclusive", F, "return best > t ? best : 0.0f;", "return best >= t ? best : 0.0f;"),
    ("abs_after_scale_sum", S,
     "f += p->rectify ? fabs(v) : v;\n                }\n                F[((size_t)k * eh + yy) * ew + xx] = f;",
     "f += v;\n                }\n                F[((size_t)k * eh + yy) * ew + xx] = p->rectify ? fabs(f) : f;"),
]


def _run_pins(tmp_path, src=None, old=None, new=None):
    """Copies the sources (planting old -> new in src if given), builds the
    copy and runs the pin tests against it; returns the pytest process."""
    for f in SRCS:
        shutil.copy(os.path.join(ROOT, "oracle", f), tmp_path / f)
    if src is not None:
        text = (tmp_path / src).read_text()
        assert text.count(old) == 1, "the planted line is no longer in %s" % src
        (tmp_path / src).write_text(text.replace(old, new))
    lib = tmp_path / "liboracle_copy.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(lib)]
                   + [str(tmp_path / f) for f in SRCS] + ["-lm"], check=True)
    env = dict(os.environ, SFOC_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider"] + PINS,
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    """The control: a copy built the same way, with nothing planted, passes
    every pin (so a failure below is the planted mistake's)."""
    r = _run_pins(tmp_path)
    assert r.returncode == 0, r.stdout[-800:]


@pytest.mark.parametrize("name,src,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pins_catch_a_planted_mistake(tmp_path, name, src, old, new):
    r = _run_pins(tmp_path, src, old, new)
    assert r.returncode != 0, "no pin caught the mutation %s:\n%s" % (name, r.stdout[-800:])
    summary = [ln for ln in r.stdout.splitlines() if " in " in ln and ("failed" in ln or "error" in ln)][-1:]
    assert summary and "failed" in summary[0] and "error" not in summary[0], r.stdout[-800:]   # a pin, not an import
