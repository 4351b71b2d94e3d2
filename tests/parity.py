"""Comparison rules shared by the GPU parity tests.

Tolerances (stated by the target: NCC within 1e-4 absolute, sub-pixel
within 0.02 px, integer offsets identical).  Where two candidates' oracle
scores are closer than 2e-4 the argmax is not unique at that precision:
the GPU's pick must then be a valid argmax, i.e. its oracle score within
2e-4 of the oracle's best.  Such near-ties are counted, never dropped: every
comparison prints its counts (and appends them to the file named by the
environment variable SFOC_PARITY_LOG, one JSON line per comparison), and the
points where the GPU took another valid argmax ("tie flips") may be at most
1 % of the valid points (at least one is allowed, for small samples).
"""
import json
import os

import numpy as np

NCC_TOL = 1e-4
SUB_TOL = 0.02
TIE = 2 * NCC_TOL
MAX_FLIP_FRAC = 0.01


def _log(stats):
    rec = dict(stats, test=os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0])
    print("parity", json.dumps(rec))
    path = os.environ.get("SFOC_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


_CACHE = {}


def cached(key, fn):
    """fn() once per key for the test session (oracle results shared by the
    forms that are compared with the same sample)."""
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


def to_np(res):
    return {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)) for k, v in res.items()}


def compare(gpu, orc, R, ncc_tol=NCC_TOL, sub_tol=SUB_TOL, oracle_maps=None, report=None):
    """Returns a dict of statistics; asserts the parity rules.  ncc_tol and
    sub_tol may be per-point arrays; offsets must agree wherever the oracle's
    best-vs-second margin exceeds twice the point's NCC tolerance."""
    g = to_np(gpu)
    n = len(orc["status"])
    assert len(g["status"]) == n
    np.testing.assert_array_equal(g["status"], orc["status"])
    ncc_tol = np.broadcast_to(np.asarray(ncc_tol, np.float64), (n,))
    sub_tol = np.broadcast_to(np.asarray(sub_tol, np.float64), (n,))
    tie = 2 * ncc_tol
    valid = np.isin(orc["status"], [0, 3])
    exact = valid & (orc["margin"] > tie)
    same = (g["dx"] == orc["dx"]) & (g["dy"] == orc["dy"])
    bad_exact = np.flatnonzero(exact & ~same)
    assert len(bad_exact) == 0, "offset mismatch at points %s" % bad_exact[:10]
    ties = np.flatnonzero(valid & ~exact & ~same)
    for k in ties:
        assert oracle_maps is not None, "near-tie at point %d needs the oracle map" % k
        mp = oracle_maps[k]
        v = mp[g["dy"][k] + R, g["dx"][k] + R]
        assert v >= orc["ncc"][k] - tie[k], (k, v, orc["ncc"][k])
    both = valid & same
    dn = np.abs(g["ncc"].astype(np.float64) - orc["ncc"])
    assert np.all(dn[both] <= ncc_tol[both]), "ncc err max %g" % (dn[both].max() if both.any() else 0)
    ds = np.maximum(np.abs(g["sub_dx"] - orc["sub_dx"]), np.abs(g["sub_dy"] - orc["sub_dy"]))
    assert np.all(ds[both] <= sub_tol[both]), "sub-pixel err max %g" % (ds[both].max() if both.any() else 0)
    stats = dict(n=n, valid=int(valid.sum()), near_ties=int((valid & ~exact).sum()), tie_flips=len(ties),
                 offsets_equal=int((valid & same).sum()),
                 ncc_err_max=float(dn[both].max()) if both.any() else 0.0,
                 sub_err_max=float(ds[both].max()) if both.any() else 0.0)
    _log(stats)
    allowed = max(1, int(MAX_FLIP_FRAC * stats["valid"]))
    assert stats["tie_flips"] <= allowed, "tie flips %d > %d allowed" % (stats["tie_flips"], allowed)
    if report is not None:
        report.update(stats)
    return stats


def subpixel_tol(omap, R, ncc_tol, base=SUB_TOL):
    """Sub-pixel tolerance implied by an NCC error e at the three samples of
    the parabola: |d delta| <= 2e (1 + 2|delta|) / (2|den| - 4e) per axis,
    den = c- - 2c0 + c+ of the oracle map; at least `base`."""
    P1 = 2 * R + 1
    i = int(np.nanargmax(omap))
    iy, ix = divmod(i, P1)
    t = base
    for (a, b_) in (((iy, ix - 1), (iy, ix + 1)), ((iy - 1, ix), (iy + 1, ix))):
        if min(a + b_) < 0 or max(a + b_) >= P1:
            continue
        cm, c0, cp = omap[a], omap[iy, ix], omap[b_]
        den = cm - 2 * c0 + cp
        if den >= 0:
            continue
        d = (cm - cp) / (2 * den)
        lim = 2 * abs(den) - 4 * ncc_tol
        t = max(t, float("inf") if lim <= 0 else 2 * ncc_tol * (1 + 2 * abs(d)) / lim)
    return t


# ---------------------------------------------------------------------------
# bf16 rounding: definition and the bound it implies for NCC
# ---------------------------------------------------------------------------

def bf16_round(x):
    """float64 -> nearest-even bfloat16 (through float32), as float64."""
    f = np.ascontiguousarray(x, np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_ulp(x):
    """Spacing of bfloat16 numbers at |x| (8 significant bits)."""
    a = np.maximum(np.abs(np.asarray(x, np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def _box(plane, m):
    """Sums over all m x m windows of a 2-D array (valid positions)."""
    P = np.zeros((plane.shape[0] + 1, plane.shape[1] + 1))
    P[1:, 1:] = plane.cumsum(0).cumsum(1)
    return P[m:, m:] - P[:-m, m:] - P[m:, :-m] + P[:-m, :-m]


def ncc_rounding_bound(S, T, cube_err=2e-5, base=NCC_TOL):
    """Per-offset bound on |dNCC| between the GPU's bf16 cube and the
    oracle's cube rounded to bf16.  The two FP32/FP64 cubes differ by at most
    `cube_err` per value, so only values within `cube_err` of a rounding
    midpoint can round differently: by one ulp where the ulp exceeds
    cube_err, by at most floor(cube_err / ulp) + 1 ulps where it does not (the
    values near zero).  A perturbation delta of a centred vector s changes
    the cosine by at most ||delta|| / ||s||, so
      bound = base + ||delta_S|| / sigma_S + ||delta_T|| / sigma_T
    with ||delta||^2 the sum of the squared moves of the ambiguous values and
    sigma the centred norms.
    S: (z, M, M) window region (FP64, unrounded), T: (z, m, m).  Returns a
    (M-m+1, M-m+1) map."""
    z, m = T.shape[0], T.shape[1]
    N = m * m * z

    def amb(v):
        lo = bf16_round(v)
        u = bf16_ulp(v)
        d = np.minimum(np.abs(v - (lo + u / 2)), np.abs(v - (lo - u / 2)))
        mv = (np.floor(cube_err / u) + 1.0) * u       # the largest move of a value within cube_err
        return np.where(d <= cube_err, mv * mv, 0.0)

    wS = amb(S)
    wT = amb(T)
    dS = np.sqrt(_box(wS.sum(0), m))                  # ||delta_S|| per offset
    dT = np.sqrt(wT.sum())
    s1 = _box(S.sum(0), m)
    s2 = _box((S * S).sum(0), m)
    sigS = np.sqrt(np.maximum(s2 - s1 * s1 / N, 1e-300))
    sigT = np.sqrt(max(((T - T.mean()) ** 2).sum(), 1e-300))
    return base + dS / sigS + dT / sigT


def flip_tolerance(Sw, T, cube_err=2e-5, base=NCC_TOL, k_sigma=6.0):
    """Tolerance at one offset for the GPU bf16 cube vs the oracle cube
    rounded to bf16.  Ambiguous values (within cube_err of a rounding
    midpoint) move independently by +-1 ulp (+-(floor(cube_err / ulp) + 1)
    ulps at most where the ulp is below cube_err); to first order the NCC
    moves by
    sum_i g_i delta_i with g the exact NCC gradient
      dNCC/ds_i = b_i/(|a||b|) - NCC a_i/|a|^2,  a = s - mean(s), b = t - mean(t)
    (and symmetrically for t), whose spread is
      sigma^2 = sum over ambiguous i of (move_i g_i)^2.
    Returns base + k_sigma * sigma.  Sw: (z, m, m) window, T: (z, m, m)."""
    a = (Sw - Sw.mean()).ravel()
    bb = (T - T.mean()).ravel()
    na, nb = np.linalg.norm(a), np.linalg.norm(bb)
    if na == 0 or nb == 0:
        return base
    ncc = float(a @ bb) / (na * nb)
    gS = bb / (na * nb) - ncc * a / (na * na)
    gT = a / (na * nb) - ncc * bb / (nb * nb)

    def w(v):
        lo = bf16_round(v)
        u = bf16_ulp(v)
        d = np.minimum(np.abs(v - (lo + u / 2)), np.abs(v - (lo - u / 2)))
        return np.where(d <= cube_err, (np.floor(cube_err / u) + 1.0) * u, 0.0).ravel()

    sig = np.sqrt(((w(Sw) * gS) ** 2).sum() + ((w(T) * gT) ** 2).sum())
    return base + k_sigma * sig


def storage_bound(S, T, base=NCC_TOL):
    """Bound on |dNCC| from storing every value in bf16 (relative error at
    most 2^-9): ||delta|| <= 2^-9 ||v||, so
      bound = base + 2^-9 (||S|| / sigma_S + ||T|| / sigma_T)  per offset."""
    z, m = T.shape[0], T.shape[1]
    N = m * m * z
    s1 = _box(S.sum(0), m)
    s2 = _box((S * S).sum(0), m)
    sigS = np.sqrt(np.maximum(s2 - s1 * s1 / N, 1e-300))
    sigT = np.sqrt(max(((T - T.mean()) ** 2).sum(), 1e-300))
    return base + 2.0 ** -9 * (np.sqrt(s2) / sigS + np.linalg.norm(T) / sigT)


def compare_maps(gmaps, omaps, bounds, valid):
    """Element-wise map check against per-point bound maps."""
    worst = 0.0
    for k in np.flatnonzero(valid):
        d = np.abs(gmaps[k].astype(np.float64) - omaps[k])
        assert np.all(d <= bounds[k]), (k, float(d.max()), float(bounds[k][np.unravel_index(d.argmax(), d.shape)]))
        worst = max(worst, float((d / bounds[k]).max()))
    return worst


# ---- BF16 form: oracle on the bf16-rounded cube, checks with derived tolerances ----

def bf16_oracle_side(orc, pair, roi=False):
    import oracle as _o

    """Oracle Eq. 8 on its cube rounded to bf16 and on the unrounded cube,
    plus per point the unrounded search region and template."""
    m, R = pair.m, pair.R
    h = orc.template_half(m)
    M = m + 2 * R
    regions = []
    if not roi:
        rc_full = orc.sfoc_roi(pair.ref)
        sc_full = orc.sfoc_roi(pair.sen)
    res_r, res_u = [], []
    for (px, py) in pair.points:
        ty0, tx0 = int(py) - h, int(px) - h
        inb = (ty0 - R >= 0 and tx0 - R >= 0 and ty0 + m + R <= pair.ref.shape[0]
               and tx0 + m + R <= pair.ref.shape[1] and ty0 + m <= pair.sen.shape[0] and tx0 + m <= pair.sen.shape[1])
        if not inb:
            regions.append(None)
            continue
        if roi:
            S = orc.sfoc_roi(pair.ref, None, ty0 - R, tx0 - R, M, M).data
            T = orc.sfoc_roi(pair.sen, None, ty0, tx0, m, m).data
        else:
            S = rc_full.data[:, ty0 - R:ty0 + m + R, tx0 - R:tx0 + m + R].copy()
            T = sc_full.data[:, ty0:ty0 + m, tx0:tx0 + m].copy()
        regions.append((S, T))

    def run(rounded):
        outs = []
        for k, (px, py) in enumerate(pair.points):
            if regions[k] is None:
                dummy = _o.CubeROI(np.zeros((12, 1, 1)), pair.ref.shape[0], pair.ref.shape[1], 0, 0)
                outs.append(orc.match(dummy, dummy, np.array([[px, py]], np.int32), m, R, want_maps=True))
                continue
            S, T = regions[k]
            ty0, tx0 = int(py) - h, int(px) - h
            Sc = bf16_round(S) if rounded else S
            Tc = bf16_round(T) if rounded else T
            rc = _o.CubeROI(np.ascontiguousarray(Sc), pair.ref.shape[0], pair.ref.shape[1], ty0 - R, tx0 - R)
            sc = _o.CubeROI(np.ascontiguousarray(Tc), pair.sen.shape[0], pair.sen.shape[1], ty0, tx0)
            outs.append(orc.match(rc, sc, np.array([[px, py]], np.int32), m, R, want_maps=True))
        return {key: np.concatenate([o[key] for o in outs]) for key in outs[0]}

    return run(True), run(False), regions


def bf16_check(g, o_r, o_u, regions, R, report):
    n = len(regions)
    bmaps = [ncc_rounding_bound(*r) if r is not None else None for r in regions]
    smaps = [storage_bound(*r) if r is not None else None for r in regions]
    tol = np.full(n, 1e-4)
    for k, reg in enumerate(regions):
        if reg is None or o_r["status"][k] not in (0, 3):
            continue
        S, T = reg
        m = T.shape[1]
        dy, dx = o_r["dy"][k] + R, o_r["dx"][k] + R
        tol[k] = flip_tolerance(S[:, dy:dy + m, dx:dx + m], T)
    sub = np.array([subpixel_tol(o_r["maps"][k], R, tol[k]) if bmaps[k] is not None else 0.02 for k in range(n)])
    st = compare(g, o_r, R, ncc_tol=tol, sub_tol=sub, oracle_maps=o_r["maps"])
    valid = np.isin(o_r["status"], [0, 3])
    if "maps" in g:
        compare_maps(g["maps"].cpu().numpy(), o_r["maps"], bmaps, valid)
    # precision report against the unrounded FP64 oracle
    gn = to_np(g)
    same = valid & (gn["dx"] == o_u["dx"]) & (gn["dy"] == o_u["dy"])
    stol = np.array([smaps[k][gn["dy"][k] + R, gn["dx"][k] + R] if smaps[k] is not None else 1.0 for k in range(n)])
    err = np.abs(gn["ncc"] - o_u["ncc"])
    assert np.all(err[same] <= stol[same]), float((err[same] - stol[same]).max())
    report.update(st, bf16_vs_fp64_offsets_equal=int(same.sum()), bf16_vs_fp64_valid=int(valid.sum()),
                  bf16_vs_fp64_ncc_err_max=float(err[same].max()) if same.any() else 0.0,
                  rounding_bound_max=float(tol[valid].max()) if valid.any() else 0.0)
    print(report)
    return st
