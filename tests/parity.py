"""Comparison rules shared by the GPU parity tests.

Tolerances (stated by the target: NCC within 1e-4 absolute, sub-pixel
within 0.02 px, integer offsets identical).  Where two candidates' oracle
scores are closer than 2e-4 the argmax is not unique at that precision:
the GPU's pick must then be a valid argmax, i.e. its oracle score within
2e-4 of the oracle's best.
"""
import numpy as np

NCC_TOL = 1e-4
SUB_TOL = 0.02
TIE = 2 * NCC_TOL


def to_np(res):
    return {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)) for k, v in res.items()}


def compare(gpu, orc, R, ncc_tol=NCC_TOL, sub_tol=SUB_TOL, oracle_maps=None, report=None):
    """Returns a dict of statistics; asserts the parity rules."""
    g = to_np(gpu)
    n = len(orc["status"])
    assert len(g["status"]) == n
    np.testing.assert_array_equal(g["status"], orc["status"])
    valid = np.isin(orc["status"], [0, 3])
    exact = valid & (orc["margin"] > TIE)
    same = (g["dx"] == orc["dx"]) & (g["dy"] == orc["dy"])
    bad_exact = np.flatnonzero(exact & ~same)
    assert len(bad_exact) == 0, "offset mismatch at points %s" % bad_exact[:10]
    ties = np.flatnonzero(valid & ~exact & ~same)
    for k in ties:
        assert oracle_maps is not None, "near-tie at point %d needs the oracle map" % k
        mp = oracle_maps[k]
        v = mp[g["dy"][k] + R, g["dx"][k] + R]
        assert v >= orc["ncc"][k] - TIE, (k, v, orc["ncc"][k])
    both = valid & same
    dn = np.abs(g["ncc"][both].astype(np.float64) - orc["ncc"][both])
    assert np.all(dn <= ncc_tol), "ncc err max %g" % (dn.max() if dn.size else 0)
    ds = np.maximum(np.abs(g["sub_dx"][both] - orc["sub_dx"][both]), np.abs(g["sub_dy"][both] - orc["sub_dy"][both]))
    assert np.all(ds <= sub_tol), "sub-pixel err max %g" % (ds.max() if ds.size else 0)
    stats = dict(n=n, valid=int(valid.sum()), near_ties=int((valid & ~exact).sum()), tie_flips=len(ties),
                 ncc_err_max=float(dn.max()) if dn.size else 0.0, sub_err_max=float(ds.max()) if ds.size else 0.0)
    if report is not None:
        report.update(stats)
    return stats
