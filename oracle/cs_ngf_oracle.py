"""Plain, slow FP64 CPU oracle for Cross-Sim-NGF's all-shift similarity.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never calls it and
shares no code with it.

What it computes (Cross-Sim-NGF, Ofverstedt, Lindblad, Sladoje):

* Eq. 1   regularised normalised gradient field n(x; A) = grad A / sqrt(|grad A|^2 + eps^2)
* Eq. 2   s_NGF = <n_A, n_B>^2
* Eq. 4-5 the masked average over the overlap, for every integer shift chi:
          CSNGF(chi) = sum_x M_A(x) M_B(x+chi) s_NGF / N(chi),  N = M_A (star) M_B
* Eq. 6-8 the same through six separable channel correlations and one mask
          correlation evaluated with FFTs (summed before one inverse transform)
* Section 3.2  B_hat = B o T_theta by trilinear interpolation; shifts with
          overlap below gamma are excluded; argmax over chi, then over rotations.
* Section 5.2  the direct algorithm: a loop over all valid shifts with the
          squared dot products summed directly.

Readings where the paper is silent (each is listed in the design notes):

1. Gradient: central differences with unit spacing; at a face the index is
   clamped, so the first sample gives (f[1] - f[0]) / 2.
2. No intensity normalisation and no smoothing before the NGF.
3. Rotated mask: M_hat(x) = [trilinear M_B(p) >= 0.5] and p inside
   [0, n-1]^3 with 1e-4 slack; outside the domain B_hat = 0, M_hat = 0.
4. Rotation: c = (n-1)/2, B_hat(x) = B(R(q)(x - c) + c), R the Hamilton
   unit-quaternion matrix built in FP64, entries within 1e-9 of -1, 0, 1
   snapped.  The sample point p and the mask decision are evaluated in FP32
   with a fixed operation order (the kernel's precision, so both sides take
   the same integer decisions); interpolated intensities are FP64 here.
5. gamma: chi is valid iff N(chi) >= max(1, ceil(gamma * min(sum M_A, sum M_hat))).
6. Shift sign: C(chi) = sum_x a(x) b(x + chi), stored at chi mod P.
7. Ties: the largest score wins; equal scores go to the smallest (z, y, x)
   shift, then the smallest rotation index.
8. Padding: full linear correlation, P >= 2n - 1 per axis.

Parity pins: every function here is checked by tests against closed forms,
invariants, library routines or brute force (tests/test_oracle_*.py).
"""
from __future__ import annotations

import math

import numpy as np

F32 = np.float32

# channel order of Eq. 6: (xx, yy, zz, xy, xz, yz); cross terms carry weight 2
CHANNEL_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))
CHANNEL_WEIGHTS = (1.0, 1.0, 1.0, 2.0, 2.0, 2.0)
MEASURES = ("squared", "unsquared")

SUPPORTED_PADS = (16, 32, 40, 64, 80, 100, 128, 160, 192, 200, 216, 256, 320, 360, 400, 512)


def auto_pad(n: int) -> int:
    """Smallest supported FFT length (2^a 3^b 5^c) >= 2n - 1 (full linear correlation)."""
    for p in SUPPORTED_PADS:
        if p >= 2 * n - 1:
            return p
    raise ValueError(f"no supported FFT length for n={n}")


# --------------------------------------------------------------------------
# Section 3.2: the rigid rotation T_theta
# --------------------------------------------------------------------------
def quat_to_rotmat(q) -> np.ndarray:
    """Hamilton unit quaternion (w, x, y, z) -> 3x3 matrix acting on (x, y, z).

    The quaternion is normalised in FP64; entries within 1e-9 of -1, 0 or 1
    are snapped so that the identity and quarter turns are exact."""
    w, x, y, z = (float(v) for v in q)
    s = math.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / s, x / s, y / s, z / s
    R = np.array([
        [1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y)],
        [2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x)],
        [2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)],
    ])
    for target in (-1.0, 0.0, 1.0):
        R[np.abs(R - target) <= 1e-9] = target
    return R


def sample_points_f32(R: np.ndarray, dims):
    """p = R (x - c) + c for every voxel x, in FP32 with a fixed order.

    d_j = float(x_j) - c_j (exact);  p_i = ((R_i0 d_0 + R_i1 d_1) + R_i2 d_2) + c_i,
    each product and sum rounded to FP32.  Returns (px, py, pz) arrays [z][y][x]."""
    nz, ny, nx = dims
    Rf = R.astype(F32)
    c = (F32((nx - 1) / 2), F32((ny - 1) / 2), F32((nz - 1) / 2))
    zz, yy, xx = np.meshgrid(np.arange(nz, dtype=F32), np.arange(ny, dtype=F32),
                             np.arange(nx, dtype=F32), indexing="ij")
    d = (xx - c[0], yy - c[1], zz - c[2])
    p = []
    for i in range(3):
        acc = Rf[i, 0] * d[0]
        acc = acc + Rf[i, 1] * d[1]
        acc = acc + Rf[i, 2] * d[2]
        acc = acc + c[i]
        p.append(acc.astype(F32))
    return p


# Section 3.2 reading of the rotated mask: sample points within this distance
# outside [0, n-1] still count as inside the domain (they sample the face).
DOMAIN_SLACK = 1e-4


def _lerp(a, b, t):
    """a + t (b - a) in FP32 (the order the mask decision is taken in)."""
    return (a + t * (b - a)).astype(F32)


def _mask_on(m):
    """The rotated mask is set where the interpolated mask reaches one half."""
    return m >= F32(0.5)


def _axis_setup(p, n):
    """Domain test, clamped base index and fraction for one axis (FP32)."""
    slack = F32(DOMAIN_SLACK)
    hi = F32(n - 1) + slack
    inside = (p >= -slack) & (p <= hi)
    pc = np.minimum(np.maximum(p, F32(0.0)), F32(n - 1))
    i0 = np.floor(pc).astype(np.int64)
    i0 = np.minimum(i0, max(n - 2, 0))
    t = (pc - i0.astype(F32)).astype(F32)
    return inside, i0, t


def resample(B: np.ndarray, MB: np.ndarray, q):
    """Section 3.2: B_hat = B o T_theta (trilinear) and the rotated mask.

    Returns (B_hat float64, M_hat uint8)."""
    dims = B.shape
    nz, ny, nx = dims
    R = quat_to_rotmat(q)
    px, py, pz = sample_points_f32(R, dims)
    ix, x0, tx = _axis_setup(px, nx)
    iy, y0, ty = _axis_setup(py, ny)
    iz, z0, tz = _axis_setup(pz, nz)
    inside = ix & iy & iz
    x1 = np.minimum(x0 + 1, nx - 1)
    y1 = np.minimum(y0 + 1, ny - 1)
    z1 = np.minimum(z0 + 1, nz - 1)

    # intensity: exact trilinear weights (FP64) at the FP32 sample point
    Bd = B.astype(np.float64)
    txd, tyd, tzd = tx.astype(np.float64), ty.astype(np.float64), tz.astype(np.float64)
    val = np.zeros(dims)
    for cz, wz in ((z0, 1 - tzd), (z1, tzd)):
        for cy, wy in ((y0, 1 - tyd), (y1, tyd)):
            for cx, wx in ((x0, 1 - txd), (x1, txd)):
                val += wz * wy * wx * Bd[cz, cy, cx]
    Bhat = np.where(inside, val, 0.0)

    # mask decision in FP32: lerp along x, then y, then z; lerp(a,b,t)=a+t*(b-a)
    M = MB.astype(F32)
    m00 = _lerp(M[z0, y0, x0], M[z0, y0, x1], tx)
    m01 = _lerp(M[z0, y1, x0], M[z0, y1, x1], tx)
    m10 = _lerp(M[z1, y0, x0], M[z1, y0, x1], tx)
    m11 = _lerp(M[z1, y1, x0], M[z1, y1, x1], tx)
    m0 = _lerp(m00, m01, ty)
    m1 = _lerp(m10, m11, ty)
    m = _lerp(m0, m1, tz)
    Mhat = (inside & _mask_on(m)).astype(np.uint8)
    return Bhat, Mhat


# --------------------------------------------------------------------------
# Eq. 1, Eq. 2, Eq. 6
# --------------------------------------------------------------------------
def gradient(V: np.ndarray):
    """Central differences with clamped indices; returns (gx, gy, gz)."""
    V = np.asarray(V, dtype=np.float64)
    out = []
    for axis in (2, 1, 0):                      # x, y, z
        n = V.shape[axis]
        up = np.take(V, np.minimum(np.arange(n) + 1, n - 1), axis=axis)
        dn = np.take(V, np.maximum(np.arange(n) - 1, 0), axis=axis)
        out.append((up - dn) / 2.0)
    return tuple(out)


def ngf(V: np.ndarray, eps: float):
    """Eq. 1: n = grad V / sqrt(|grad V|^2 + eps^2); returns (nx, ny, nz)."""
    gx, gy, gz = gradient(V)
    inv = 1.0 / np.sqrt(gx * gx + gy * gy + gz * gz + float(eps) ** 2)
    return gx * inv, gy * inv, gz * inv


def s_ngf(nA, nB, measure="squared"):
    """Eq. 2 (squared dot product of two NGF vectors, voxel-wise) or Eq. 3
    (the plain dot product) for measure="unsquared"."""
    d = nA[0] * nB[0] + nA[1] * nB[1] + nA[2] * nB[2]
    return d * d if measure == "squared" else d


def channels(V: np.ndarray, M: np.ndarray, eps: float, measure="squared"):
    """Eq. 6 channels times the mask, M * (nx^2, ny^2, nz^2, nx ny, nx nz, ny nz),
    or for Eq. 3 the three components M * (nx, ny, nz)."""
    n = ngf(V, eps)
    m = np.asarray(M, dtype=np.float64)
    if measure == "unsquared":
        return [m * n[i] for i in range(3)]
    return [m * n[i] * n[j] for (i, j) in CHANNEL_PAIRS]


def channel_weights(measure="squared"):
    return CHANNEL_WEIGHTS if measure == "squared" else (1.0, 1.0, 1.0)


def overlap_threshold(sumA: int, sumB: int, gamma: float) -> int:
    """Section 3.2 minimum overlap: max(1, ceil(gamma * min(sum M_A, sum M_hat)))."""
    return max(1, int(math.ceil(float(gamma) * float(min(int(sumA), int(sumB))))))


# --------------------------------------------------------------------------
# Eq. 5 by the direct algorithm (Section 5.2)
# --------------------------------------------------------------------------
def _shift_slices(chi, dims_a, dims_b):
    sa, sb = [], []
    for c, na, nb in zip(chi, dims_a, dims_b):
        lo = max(0, -c)
        hi = min(na, nb - c)
        if hi <= lo:
            return None
        sa.append(slice(lo, hi))
        sb.append(slice(lo + c, hi + c))
    return tuple(sa), tuple(sb)


def csngf_direct(A, MA, Bhat, Mhat, eps, gamma, chis=None, measure="squared"):
    """Eq. 5 evaluated shift by shift: returns (score map, overlap map).

    The maps cover chi in [-(n-1), n-1] per axis (array index chi + n - 1);
    invalid shifts hold -inf in the score map.  If ``chis`` is given, only
    those shifts are evaluated (others stay -inf / 0)."""
    dims = A.shape
    nA = ngf(A, eps)
    nB = ngf(Bhat, eps)
    ma = np.asarray(MA, dtype=np.float64)
    mb = np.asarray(Mhat, dtype=np.float64)
    thr = overlap_threshold(int(ma.sum()), int(mb.sum()), gamma)
    shape = tuple(2 * n - 1 for n in dims)
    score = np.full(shape, -np.inf)
    count = np.zeros(shape, dtype=np.int64)
    if chis is None:
        chis = np.stack(np.meshgrid(*[np.arange(-(n - 1), n) for n in dims],
                                    indexing="ij"), axis=-1).reshape(-1, 3)
    for chi in chis:
        chi = tuple(int(c) for c in chi)
        idx = tuple(c + n - 1 for c, n in zip(chi, dims))
        sl = _shift_slices(chi, dims, dims)
        if sl is None:
            continue
        sa, sb = sl
        w = ma[sa] * mb[sb]
        N = int(round(w.sum()))
        count[idx] = N
        if N < thr:
            continue
        d = nA[0][sa] * nB[0][sb] + nA[1][sa] * nB[1][sb] + nA[2][sa] * nB[2][sb]
        val = d * d if measure == "squared" else d
        score[idx] = float((w * val).sum()) / N
    return score, count


# --------------------------------------------------------------------------
# Eq. 6-8: the frequency-domain form
# --------------------------------------------------------------------------
def correlate_fft(a, b, pad):
    """C(chi) = sum_x a(x) b(x + chi) for chi in [-(n-1), n-1]^3 via rfftn/irfftn."""
    dims = a.shape
    Fa = np.fft.rfftn(a, s=pad, axes=(0, 1, 2))
    Fb = np.fft.rfftn(b, s=pad, axes=(0, 1, 2))
    c = np.fft.irfftn(np.conj(Fa) * Fb, s=pad, axes=(0, 1, 2))
    return _gather_shifts(c, dims, pad)


def _gather_shifts(c, dims, pad):
    idx = [np.mod(np.arange(-(n - 1), n), p) for n, p in zip(dims, pad)]
    return c[np.ix_(*idx)]


def csngf_fft(A, MA, Bhat, Mhat, eps, gamma, pad=None, measure="squared"):
    """Eq. 6-8: six weighted channel correlations summed in the spectrum, one
    inverse FFT, divided by the mask correlation N (Eq. 5).  With
    measure="unsquared" the three Eq. 3 component correlations instead."""
    dims = A.shape
    if pad is None:
        pad = tuple(auto_pad(n) for n in dims)
    pad = tuple(int(p) for p in pad)
    a = channels(A, MA, eps, measure)
    b = channels(Bhat, Mhat, eps, measure)
    acc = None
    for w, ac, bc in zip(channel_weights(measure), a, b):
        term = w * np.conj(np.fft.rfftn(ac, s=pad, axes=(0, 1, 2))) * np.fft.rfftn(bc, s=pad, axes=(0, 1, 2))
        acc = term if acc is None else acc + term
    X = _gather_shifts(np.fft.irfftn(acc, s=pad, axes=(0, 1, 2)), dims, pad)
    ma = np.asarray(MA, dtype=np.float64)
    mb = np.asarray(Mhat, dtype=np.float64)
    Nf = correlate_fft(ma, mb, pad)
    N = np.rint(Nf).astype(np.int64)
    thr = overlap_threshold(int(ma.sum()), int(mb.sum()), gamma)
    score = np.full(X.shape, -np.inf)
    ok = N >= thr
    score[ok] = X[ok] / N[ok]
    return score, N


def best_of_map(score):
    """argmax over chi with the tie rule; returns (score, (cz, cy, cx)) or
    (-inf, (0, 0, 0)) when no shift is valid."""
    if not np.any(np.isfinite(score)):
        return -np.inf, (0, 0, 0)
    flat = int(np.argmax(score))          # first occurrence = smallest (z, y, x)
    idx = np.unravel_index(flat, score.shape)
    dims = tuple((s + 1) // 2 for s in score.shape)
    chi = tuple(int(i) - (n - 1) for i, n in zip(idx, dims))
    return float(score[idx]), chi


def score_map(A, MA, B, MB, q, eps=1e-5, gamma=0.5, pad=None, form="fft", measure="squared"):
    """Full score map for one rotation q (Section 3.2 then Eq. 5)."""
    Bhat, Mhat = resample(B, MB, q)
    if form == "direct":
        return csngf_direct(A, MA, Bhat, Mhat, eps, gamma, measure=measure)
    return csngf_fft(A, MA, Bhat, Mhat, eps, gamma, pad, measure=measure)


def score_rotations(A, MA, B, MB, quats, eps=1e-5, gamma=0.5, pad=None, form="fft",
                    measure="squared"):
    """Per rotation: best score over chi and its shift (z, y, x)."""
    scores, shifts = [], []
    for q in quats:
        s, _ = score_map(A, MA, B, MB, q, eps, gamma, pad, form, measure)
        b, chi = best_of_map(s)
        scores.append(b)
        shifts.append(chi)
    return np.array(scores), np.array(shifts, dtype=np.int64).reshape(-1, 3)


def align(A, MA, B, MB, quats, eps=1e-5, gamma=0.5, pad=None):
    """Max over rotations of the per-rotation best (Fig. 1): (score, r, shift)."""
    scores, shifts = score_rotations(A, MA, B, MB, quats, eps, gamma, pad)
    if not np.any(np.isfinite(scores)):
        return -np.inf, -1, (0, 0, 0)
    r = int(np.argmax(scores))
    return float(scores[r]), r, tuple(int(v) for v in shifts[r])
