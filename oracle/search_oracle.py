"""FP64 CPU reference of the global search driver (Section 3.2).

TEST INFRASTRUCTURE ONLY (like cs_ngf_oracle): imported by tests, never by the
product path.

The pyramid: level k smooths A and B with a Gaussian of sigma_k voxels
(scipy.ndimage.gaussian_filter1d along z, y, x, truncated at 4 sigma, faces
clamped: mode "nearest"), keeps every d_k-th voxel, samples the masks at the
same voxels, and scores the starting points plus a_k random rotations (a
uniformly chosen starting point plus U(-u_k, u_k) degrees on each Euler angle:
about x, then the resulting y, then the resulting z).  The best p_{k+1}
rotations (stable order on equal scores) start the next level.  Random numbers
come from SplitMix64, as published by Vigna, so the same candidates can be
replayed.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import ndimage

from . import cs_ngf_oracle as O

MASK64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


def euler_to_quat(e_deg):
    """Rotation about x, then the resulting y, then the resulting z: the
    product qx * qy * qz of the three half-angle quaternions."""
    h = [math.radians(v) / 2 for v in e_deg]
    qx = np.array([math.cos(h[0]), math.sin(h[0]), 0.0, 0.0])
    qy = np.array([math.cos(h[1]), 0.0, math.sin(h[1]), 0.0])
    qz = np.array([math.cos(h[2]), 0.0, 0.0, math.sin(h[2])])
    return hamilton(hamilton(qx, qy), qz)


def hamilton(a, b):
    w1, v1 = a[0], np.asarray(a[1:])
    w2, v2 = b[0], np.asarray(b[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


def level_volume(V, M, sigma, d):
    V = np.asarray(V, dtype=np.float64)
    if sigma > 0:
        for axis in range(3):
            V = ndimage.gaussian_filter1d(V, sigma, axis=axis, mode="nearest", truncate=4.0)
    return V[::d, ::d, ::d], (np.asarray(M)[::d, ::d, ::d] != 0).astype(np.uint8)


def global_align(A, MA, B, MB, schedule, seed, eps=1e-5, gamma=0.5, start=(0.0, 0.0, 0.0)):
    """schedule: list of (sigma, d, u_deg, a, p) per level, p being that
    level's number of starting points (the paper's p_k = |Theta_k|; the first
    level starts from `start` alone).  Level k keeps its best p_{k+1}
    rotations for level k + 1.  Returns (score, euler_deg, shift_full_res,
    level_best, candidates_per_level)."""
    rng = SplitMix64(seed)
    starts = [tuple(float(v) for v in start)]
    level_best, cands_log = [], []
    result = None
    for k, (sigma, d, u, a, _p) in enumerate(schedule):
        Ak, MAk = level_volume(A, MA, sigma, d)
        Bk, MBk = level_volume(B, MB, sigma, d)
        cand = list(starts)
        for _ in range(a):
            pick = min(len(starts) - 1, int(rng.uniform() * len(starts)))
            e = list(starts[pick])
            for ax in range(3):
                e[ax] += (2.0 * rng.uniform() - 1.0) * u
            cand.append(tuple(e))
        quats = [euler_to_quat(e) for e in cand]
        scores, shifts = O.score_rotations(Ak, MAk, Bk, MBk, quats, eps=eps, gamma=gamma)
        order = sorted(range(len(cand)), key=lambda i: (not np.isfinite(scores[i]),
                                                         -scores[i] if np.isfinite(scores[i]) else 0.0, i))
        level_best.append(float(scores[order[0]]))
        cands_log.append((cand, scores, shifts))
        keep = schedule[k + 1][4] if k + 1 < len(schedule) else 1
        starts = [cand[i] for i in order[:keep]]
        b = order[0]
        result = (float(scores[b]), cand[b], tuple(int(v) * d for v in shifts[b]))
    return result[0], result[1], result[2], level_best, cands_log
