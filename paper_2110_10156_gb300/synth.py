"""Seeded synthetic volume pairs shaped like the paper's brain blocks.

This module only builds inputs. It holds none of the alignment method's
arithmetic (no NGF, no trilinear resample, no correlation), so that both the
FP64 oracle and the CUDA path can be fed from it without sharing code.

The paper evaluates on 151^3 blocks of the CERMEP-IDB-MRXFDG brain volumes
(Section 4), displaced by a random rotation and an axis-aligned shift of up to
30 voxels and resampled with bicubic interpolation.  That dataset is not
available here, so the pairs below stand in for it:

* A is a sum of randomly oriented solid ellipsoids with intensities in U[0,1],
  Gaussian-blurred.
* B is A moved by a known rotation ``q_true`` and integer shift ``t``, sampled
  with cubic splines (the paper's data construction also uses a cubic kernel,
  distinct from the method's trilinear resample), then pushed through a
  random non-monotone 8-knot piecewise-linear intensity map (a multimodal
  stand-in: one tissue dark in one modality and bright in the other) and
  N(0, 0.01) noise.

Geometry convention (shared with the library's documentation):
arrays are indexed ``[z][y][x]`` with x contiguous; vectors are ordered
(x, y, z); the rotation centre is ``c = (n - 1) / 2`` per axis.  B is built as
``B(y) = A(R_true^T (y - c) + c - t)`` so that the method, which resamples
``B_hat(x) = B(R(q)(x - c) + c)``, recovers shift ``chi = t`` at ``q = q_true``.
Shifts are reported in array order (z, y, x).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy import ndimage
from scipy.spatial.transform import Rotation


@dataclass
class Pair:
    A: np.ndarray            # float32 [nz][ny][nx]
    MA: np.ndarray           # uint8 0/1
    B: np.ndarray            # float32
    MB: np.ndarray           # uint8 0/1
    quats: np.ndarray        # float64 [R][4] (w, x, y, z), unit
    true_index: int          # index of q_true in quats
    q_true: np.ndarray       # (w, x, y, z)
    t_zyx: tuple             # true shift in array order
    meta: dict = field(default_factory=dict)


def random_quaternions(rng: np.random.Generator, k: int) -> np.ndarray:
    """Uniform random unit quaternions (w, x, y, z) by Shoemake's subgroup
    algorithm (Graphics Gems III, 1992)."""
    u1, u2, u3 = rng.random(k), rng.random(k), rng.random(k)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    q = np.stack([w, x, y, z], axis=1)
    q[q[:, 0] < 0] *= -1.0
    return q


def axis_angle_quaternion(axis, angle_rad) -> np.ndarray:
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    h = 0.5 * angle_rad
    return np.array([np.cos(h), *(np.sin(h) * axis)])


def _scipy_matrix(q_wxyz) -> np.ndarray:
    """3x3 matrix acting on (x, y, z) vectors, via scipy's own routine."""
    w, x, y, z = q_wxyz
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def ellipsoid_phantom(rng, dims, count, rmin, rmax, sigma) -> np.ndarray:
    nz, ny, nx = dims
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1).astype(np.float64)   # (x, y, z)
    vol = np.zeros(dims, dtype=np.float64)
    n = np.array([nx, ny, nz], dtype=np.float64)
    orients = random_quaternions(rng, count)
    for k in range(count):
        centre = rng.uniform(0.25 * n, 0.75 * n)
        radii = rng.uniform(rmin, rmax, size=3)
        Rk = _scipy_matrix(orients[k])
        local = (pts - centre) @ Rk            # rows: R^T (p - centre)
        inside = np.sum((local / radii) ** 2, axis=-1) <= 1.0
        vol[inside] += rng.random()
    if sigma > 0:
        vol = ndimage.gaussian_filter(vol, sigma)
    return vol.astype(np.float32)


def move_volume(V, q_wxyz, t_xyz, order) -> np.ndarray:
    """out(y) = V(R^T (y - c) + c - t), cubic (order 3) or nearest (order 0)."""
    nz, ny, nx = V.shape
    c = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2])
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx, yy, zz], axis=-1).reshape(-1, 3).astype(np.float64)
    R = _scipy_matrix(q_wxyz)
    src = (pts - c) @ R + c - np.asarray(t_xyz, dtype=np.float64)   # R^T (p - c)
    coords = np.stack([src[:, 2], src[:, 1], src[:, 0]])            # (z, y, x)
    out = ndimage.map_coordinates(V.astype(np.float64), coords, order=order,
                                  mode="constant", cval=0.0, prefilter=(order > 1))
    return out.reshape(V.shape)


def nonmonotone_map(rng, lo, hi, knots=8):
    xs = np.linspace(lo, hi, knots)
    while True:
        ys = rng.random(knots)
        d = np.diff(ys)
        if np.any(d > 0) and np.any(d < 0):
            return xs, ys


def make_pair(seed: int, dims, n_ell: int, rmin: float, rmax: float,
              max_angle_deg: float, max_shift: int, n_rot: int,
              masks: str = "full", include_identity: bool = False,
              sigma: float | None = None, noise: float = 0.01) -> Pair:
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = tuple(int(d) for d in dims)
    if sigma is None:
        sigma = max(1.0, max(dims) / 75.0)
    A = ellipsoid_phantom(rng, dims, n_ell, rmin, rmax, sigma)
    ax = rng.normal(size=3)
    ang = np.deg2rad(rng.uniform(0.3, 1.0) * max_angle_deg)
    q_true = axis_angle_quaternion(ax, ang)
    t_xyz = rng.integers(-max_shift, max_shift + 1, size=3)
    Bgeo = move_volume(A, q_true, t_xyz, order=3)
    xs, ys = nonmonotone_map(rng, float(Bgeo.min()), float(Bgeo.max()))
    B = np.interp(Bgeo, xs, ys) + rng.normal(0.0, noise, size=Bgeo.shape)
    if masks == "full":
        MA = np.ones(dims, dtype=np.uint8)
        MB = np.ones(dims, dtype=np.uint8)
    else:
        MA = (A > 0.05 * float(A.max())).astype(np.uint8)
        MB = (move_volume(MA.astype(np.float64), q_true, t_xyz, order=0) > 0.5).astype(np.uint8)
    head = [q_true] + ([np.array([1.0, 0.0, 0.0, 0.0])] if include_identity else [])
    rest = random_quaternions(rng, max(0, n_rot - len(head)))
    if include_identity:
        quats = np.concatenate([np.stack(head), rest])
        true_index = 0
    else:
        true_index = int(rng.integers(0, n_rot))
        quats = np.insert(rest, true_index, q_true, axis=0)
    return Pair(A=A, MA=MA, B=B.astype(np.float32), MB=MB, quats=quats,
                true_index=true_index, q_true=q_true,
                t_zyx=(int(t_xyz[2]), int(t_xyz[1]), int(t_xyz[0])),
                meta=dict(seed=seed, dims=dims, angle_deg=float(np.rad2deg(ang))))


def config_pair(config: int, n_rot: int | None = None) -> Pair:
    """The seeded workloads (seed = 1000 + config number).

    0: 32^3, 12 ellipsoids r 3-10, shift <= 6, full masks, 8 rotations
       (q_true, identity, 6 random), 64^3 FFT.
    1: 150^3, 40 ellipsoids r 5-30, angle <= 30 deg, shift <= 20,
       thresholded masks, 1000 rotations, 320^3 FFT.
    4: 256^3, 48 ellipsoids r 8-50, 5000 rotations, 512^3 FFT.
    """
    if config == 0:
        return make_pair(1000, (32, 32, 32), 12, 3, 10, 45.0, 6,
                         8 if n_rot is None else n_rot, masks="full",
                         include_identity=True)
    if config == 1:
        return make_pair(1001, (150, 150, 150), 40, 5, 30, 30.0, 20,
                         1000 if n_rot is None else n_rot, masks="threshold")
    if config == 4:
        return make_pair(1004, (256, 256, 256), 48, 8, 50, 30.0, 20,
                         5000 if n_rot is None else n_rot, masks="threshold")
    raise ValueError(f"unknown config {config}")


def small_pair(seed: int, dims, n_rot: int = 4, masks: str = "threshold",
               max_shift: int = 2, max_angle_deg: float = 30.0) -> Pair:
    """Small random pair for parity tests (sizes the oracle finishes fast)."""
    n = max(dims)
    return make_pair(seed, dims, max(3, n // 4), max(1.5, n / 10), max(2.5, n / 4),
                     max_angle_deg, max_shift, n_rot, masks=masks,
                     include_identity=True, sigma=1.0)
