"""Sharding one registration job over several ranks (one process per GPU).

The path needs no exchange while it computes: image pairs are independent,
points are independent given the two cubes, and the SFOC cube is local
(every value depends on the input within HALO pixels, the derivative radius
plus three times the smoothing radius of the paper's parameters).  So a job
splits either by pairs (a batch) or, for one large pair, by bands of rows,
and the only collective is a final gather of the per-point results.

Host logic only (index arithmetic and the gather); every rank runs the
library on its own shard.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# input rows one SFOC value depends on, either side: derivative radius
# ceil(3 * 1.5) = 5 plus three times the smoothing radius ceil(3 * 1.5) = 5
HALO = 20


def template_half(m: int) -> int:
    """Rows of a template above its centre (odd m: (m-1)/2; even m: m/2)."""
    return (m - 1) // 2 if m % 2 else m // 2


def pair_cost(n_points: int, m: int, R: int, pixels: int) -> float:
    """Relative work of one pair: its correlation (m^2 (2R+1)^2 per point)
    plus its SFOC build (about 2e3 operations per pixel)."""
    return float(n_points) * m * m * (2 * R + 1) ** 2 + 2.0e3 * pixels


def shard_pairs(costs, world: int):
    """Pairs to ranks, largest first to the least loaded rank (the longest-
    processing-time rule); returns one sorted list of pair indices per rank."""
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: -costs[k]):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(v) for v in out]


@dataclass
class Band:
    y_lo: int          # rows [y_lo, y_hi) of the image hold this band's point centres
    y_hi: int
    s0: int            # rows [s0, s1) of the reference and sensed images this band reads
    s1_ref: int
    s1_sen: int
    points: np.ndarray  # indices of its points in the job's point list


def row_bands(H_ref: int, H_sen: int, points: np.ndarray, m: int, R: int, world: int, halo: int = HALO):
    """One pair split into `world` bands of point rows.  Band r takes the
    points whose centre row lies in [r H / world, (r + 1) H / world) (H the
    sensed height) and reads the image rows its templates and windows use
    plus `halo` rows either side, clipped to the images: every cube value its
    points read is then computed from the same inputs as on the whole image
    (clamped borders only where the image itself ends)."""
    h = template_half(m)
    ys = np.asarray(points)[:, 1]
    out = []
    for r in range(world):
        y_lo, y_hi = r * H_sen // world, (r + 1) * H_sen // world
        idx = np.flatnonzero((ys >= y_lo) & (ys < y_hi))
        s0 = max(0, y_lo - h - R - halo)
        top = y_hi - 1 - h + m + R + halo  # one past the last row a point of the band reads
        out.append(Band(y_lo, y_hi, s0, min(H_ref, top), min(H_sen, top), idx))
    return out


def band_inputs(ref: np.ndarray, sen: np.ndarray, points: np.ndarray, band: Band):
    """The band's image slices and its points in slice coordinates."""
    pts = np.asarray(points)[band.points].copy()
    pts[:, 1] -= band.s0
    return (np.ascontiguousarray(ref[band.s0:band.s1_ref]), np.ascontiguousarray(sen[band.s0:band.s1_sen]),
            np.ascontiguousarray(pts, dtype=np.int32))


def gather_results(dist, rank: int, world: int, n_total: int, indices, results, width: int = 6):
    """The final collective: every rank's (indices, results rows) to rank 0,
    which returns the job's (n_total, width) result array in the original
    point order (other ranks return None).  `dist` None = one rank."""
    results = np.asarray(results)
    if dist is None:
        full = np.zeros((n_total, width), dtype=results.dtype)
        full[np.asarray(indices, np.int64)] = results
        return full
    parts = [None] * world if rank == 0 else None
    dist.gather_object((np.asarray(indices, np.int64), results), parts, dst=0)
    if rank != 0:
        return None
    full = np.zeros((n_total, width), dtype=results.dtype)
    seen = np.zeros(n_total, dtype=np.int64)
    for idx, res in parts:
        full[idx] = res
        seen[idx] += 1
    if not np.all(seen == 1):
        raise RuntimeError("the ranks' shards do not cover every point exactly once")
    return full
