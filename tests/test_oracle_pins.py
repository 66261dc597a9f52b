"""Pins for the FP64 oracle, against things other than itself.

Each test checks the oracle against a closed form, an invariant the paper
states, a library routine, or brute force on tiny inputs.  The mutation tests
at the end plant plausible mistakes in the oracle (on the CPU) and check that
at least one pin catches each of them.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rand_case(seed, dims, mask_frac=0.8):
    rng = np.random.default_rng(seed)
    A = rng.random(dims)
    B = rng.random(dims)
    MA = (rng.random(dims) < mask_frac).astype(np.uint8)
    MB = (rng.random(dims) < mask_frac).astype(np.uint8)
    return A, MA, B, MB


# ---------------------------------------------------------------- brute force
def brute_csngf(A, MA, B, MB, eps, gamma):
    """Eq. 1, 2 and 5 with scalar loops only (independent of the oracle)."""
    nz, ny, nx = A.shape

    def grad(V, z, y, x):
        def at(zz, yy, xx):
            return V[min(max(zz, 0), nz - 1), min(max(yy, 0), ny - 1), min(max(xx, 0), nx - 1)]
        return ((at(z, y, x + 1) - at(z, y, x - 1)) / 2,
                (at(z, y + 1, x) - at(z, y - 1, x)) / 2,
                (at(z + 1, y, x) - at(z - 1, y, x)) / 2)

    def nvec(V, z, y, x):
        g = grad(V, z, y, x)
        den = math.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2 + eps ** 2)
        return [v / den for v in g]

    sumA, sumB = int(MA.sum()), int(MB.sum())
    thr = max(1, math.ceil(gamma * min(sumA, sumB)))
    out = {}
    for cz in range(-(nz - 1), nz):
        for cy in range(-(ny - 1), ny):
            for cx in range(-(nx - 1), nx):
                num, N = 0.0, 0
                for z in range(nz):
                    for y in range(ny):
                        for x in range(nx):
                            zb, yb, xb = z + cz, y + cy, x + cx
                            if not (0 <= zb < nz and 0 <= yb < ny and 0 <= xb < nx):
                                continue
                            if MA[z, y, x] and MB[zb, yb, xb]:
                                a = nvec(A, z, y, x)
                                b = nvec(B, zb, yb, xb)
                                d = a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
                                num += d * d
                                N += 1
                out[(cz, cy, cx)] = (num / N if N >= thr else -np.inf, N)
    return out


def test_direct_matches_brute_force_tiny():
    A, MA, B, MB = rand_case(1, (3, 4, 3))
    eps, gamma = 0.05, 0.5
    s, N = O.csngf_direct(A, MA, B, MB, eps, gamma)
    ref = brute_csngf(A, MA, B, MB, eps, gamma)
    for chi, (sv, nv) in ref.items():
        idx = tuple(c + n - 1 for c, n in zip(chi, A.shape))
        assert N[idx] == nv
        if np.isfinite(sv):
            assert s[idx] == pytest.approx(sv, rel=1e-12, abs=1e-14)
        else:
            assert not np.isfinite(s[idx])


@pytest.mark.parametrize("dims,seed", [((6, 6, 6), 2), ((5, 7, 6), 3), ((8, 8, 8), 4)])
def test_fft_form_equals_direct_all_shifts(dims, seed):
    A, MA, B, MB = rand_case(seed, dims)
    s_d, N_d = O.csngf_direct(A, MA, B, MB, 1e-3, 0.5)
    s_f, N_f = O.csngf_fft(A, MA, B, MB, 1e-3, 0.5)
    assert np.array_equal(N_d, N_f)
    fin = np.isfinite(s_d)
    assert np.array_equal(fin, np.isfinite(s_f))
    np.testing.assert_allclose(s_f[fin], s_d[fin], rtol=1e-10, atol=1e-12)


def test_fft_form_equals_direct_nonminimal_pad():
    A, MA, B, MB = rand_case(5, (6, 5, 7))
    s_d, _ = O.csngf_direct(A, MA, B, MB, 1e-3, 0.3)
    s_f, _ = O.csngf_fft(A, MA, B, MB, 1e-3, 0.3, pad=(16, 32, 16))
    fin = np.isfinite(s_d)
    np.testing.assert_allclose(s_f[fin], s_d[fin], rtol=1e-10, atol=1e-12)


# -------------------------------------------------------------- closed forms
def test_overlap_of_full_boxes_is_product():
    dims = (5, 6, 7)
    one = np.ones(dims)
    N = np.rint(O.correlate_fft(one, one, (16, 16, 16))).astype(int)
    for idx in itertools.product(*[range(2 * n - 1) for n in dims]):
        chi = [i - (n - 1) for i, n in zip(idx, dims)]
        assert N[idx] == np.prod([n - abs(c) for n, c in zip(dims, chi)])


def test_delta_fixes_shift_sign():
    dims = (6, 6, 6)
    a = np.zeros(dims)
    b = np.zeros(dims)
    a[1, 2, 3] = 1.0
    b[4, 1, 5] = 1.0                      # b = a moved by t = (+3, -1, +2)
    C = O.correlate_fft(a, b, (16, 16, 16))
    idx = np.unravel_index(np.argmax(C), C.shape)
    chi = tuple(int(i) - (n - 1) for i, n in zip(idx, dims))
    assert chi == (3, -1, 2)
    assert C[idx] == pytest.approx(1.0, abs=1e-12)
    assert np.sum(np.abs(C) > 1e-9) == 1


def test_numpy_fft_matches_definition():
    rng = np.random.default_rng(7)
    for L in (5, 8, 16, 20, 25, 64):
        x = rng.normal(size=L) + 1j * rng.normal(size=L)
        k = np.arange(L)
        W = np.exp(-2j * np.pi * np.outer(k, k) / L)
        np.testing.assert_allclose(np.fft.fft(x), W @ x, rtol=1e-11, atol=1e-11)


def test_gradient_and_ngf_on_linear_ramp():
    dims = (6, 7, 8)
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in dims], indexing="ij")
    a, u = 3e-5, np.array([0.6, 0.0, 0.8])            # direction (x, y, z)
    V = a * (u[0] * xx + u[1] * yy + u[2] * zz)
    gx, gy, gz = O.gradient(V)
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(gx[inner], a * u[0], rtol=1e-9)
    np.testing.assert_allclose(gz[inner], a * u[2], rtol=1e-9)
    # face: one-sided difference halved
    np.testing.assert_allclose(gx[:, :, 0], a * u[0] / 2, rtol=1e-9)
    n = O.ngf(V, 1e-5)
    scale = a / math.sqrt(a * a + 1e-10)
    np.testing.assert_allclose(n[0][inner], u[0] * scale, rtol=1e-9)
    np.testing.assert_allclose(n[2][inner], u[2] * scale, rtol=1e-9)


def test_s_ngf_parallel_antiparallel_orthogonal():
    e = [np.array([1.0]), np.array([0.0]), np.array([0.0])]
    assert O.s_ngf(e, e)[0] == 1.0
    assert O.s_ngf(e, [-e[0], e[1], e[2]])[0] == 1.0
    assert O.s_ngf(e, [e[1], e[0], e[2]])[0] == 0.0


def test_scores_bounded_in_unit_interval():
    A, MA, B, MB = rand_case(11, (7, 7, 7))
    s, _ = O.csngf_fft(A, MA, B, MB, 1e-3, 0.5)
    fin = s[np.isfinite(s)]
    assert fin.size > 0
    assert fin.min() >= -1e-12 and fin.max() <= 1 + 1e-12


def test_threshold_closed_form():
    assert O.overlap_threshold(100, 51, 0.5) == 26
    assert O.overlap_threshold(100, 50, 0.5) == 25
    assert O.overlap_threshold(0, 50, 0.5) == 1
    assert O.overlap_threshold(7, 9, 1.0) == 7


# ------------------------------------------------------------- rotations
def test_quaternion_matrix_matches_scipy():
    rng = np.random.default_rng(3)
    for q in synth.random_quaternions(rng, 20):
        R = O.quat_to_rotmat(q)
        Rs = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, Rs, atol=1e-12)


def quarter_turn(axis):
    q = synth.axis_angle_quaternion(np.eye(3)[axis], np.pi / 2)
    R = np.rint(Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()).astype(int)
    return q, R


def permute_volume(V, R):
    """out(y) = V(R^T (y - c) + c) by integer index arithmetic (cubes)."""
    n = V.shape[0]
    out = np.empty_like(V)
    c2 = n - 1                                   # 2c
    for zb, yb, xb in itertools.product(range(n), repeat=3):
        d2 = np.array([2 * xb - c2, 2 * yb - c2, 2 * zb - c2])
        s2 = R.T @ d2 + c2
        xa, ya, za = (s2 // 2)
        out[zb, yb, xb] = V[za, ya, xa]
    return out


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quarter_turn_resample_is_exact_permutation(axis):
    rng = np.random.default_rng(axis)
    n = 7
    A = rng.random((n, n, n))
    M = (rng.random((n, n, n)) < 0.7).astype(np.uint8)
    q, R = quarter_turn(axis)
    assert np.array_equal(O.quat_to_rotmat(q), R.astype(float))
    B = permute_volume(A, R)
    MB = permute_volume(M, R)
    Bh, Mh = O.resample(B, MB, q)
    assert np.array_equal(Bh, A)
    assert np.array_equal(Mh, M)
    s_rot, _ = O.score_map(A, M, B, MB, q, eps=1e-3)
    s_self, _ = O.csngf_fft(A, M, A, M, 1e-3, 0.5)
    np.testing.assert_array_equal(s_rot, s_self)


def test_identity_resample_is_exact():
    A, MA, B, MB = rand_case(4, (5, 6, 7))
    Bh, Mh = O.resample(B, MB, (1.0, 0.0, 0.0, 0.0))
    assert np.array_equal(Bh, B)
    assert np.array_equal(Mh, MB)


def test_trilinear_reproduces_affine_functions():
    dims = (9, 10, 11)
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for n in dims], indexing="ij")
    coef = np.array([0.3, -1.1, 0.7])
    B = 2.0 + coef[0] * xx + coef[1] * yy + coef[2] * zz
    q = synth.axis_angle_quaternion([1.0, 2.0, -0.5], 0.4)
    Bh, Mh = O.resample(B, np.ones(dims, np.uint8), q)
    R = O.quat_to_rotmat(q)
    px, py, pz = O.sample_points_f32(R, dims)
    inside = Mh.astype(bool)
    expect = 2.0 + coef[0] * px.astype(float) + coef[1] * py.astype(float) + coef[2] * pz.astype(float)
    assert inside.sum() > 0.3 * B.size
    np.testing.assert_allclose(Bh[inside], expect[inside], rtol=0, atol=1e-9)
    assert np.all(Bh[~inside & (Mh == 0)][:0] == 0)


def test_sample_points_rotate_about_centre():
    dims = (9, 9, 9)
    q = synth.axis_angle_quaternion([0, 0, 1], np.pi / 2)     # 90 deg about z
    px, py, pz = O.sample_points_f32(O.quat_to_rotmat(q), dims)
    # x-axis unit step from the centre maps to +y: p(c + e_x) = c + R e_x = c + e_y
    assert (px[4, 4, 5], py[4, 4, 5], pz[4, 4, 5]) == (4.0, 5.0, 4.0)


# ----------------------------------------------------- invariants of Eq. 2
def test_negated_intensity_gives_identical_scores():
    A, MA, B, MB = rand_case(8, (6, 7, 6))
    s1, _ = O.csngf_fft(A, MA, B, MB, 1e-3, 0.5)
    s2, _ = O.csngf_fft(A, MA, -B, MB, 1e-3, 0.5)
    np.testing.assert_array_equal(s1, s2)


def test_integer_shift_at_identity_recovers_shift_and_closed_form():
    rng = np.random.default_rng(21)
    n, t = 14, (2, -1, 3)                         # (z, y, x)
    A = np.zeros((n, n, n))
    core = slice(5, 9)
    A[core, core, core] = rng.random((4, 4, 4)) + 0.5
    B = np.roll(A, t, axis=(0, 1, 2))             # B(y) = A(y - t), zero borders
    M = np.ones_like(A, dtype=np.uint8)
    s, N = O.score_map(A, M, B, M, (1, 0, 0, 0), eps=1e-5)
    best, chi = O.best_of_map(s)
    assert chi == t
    gx, gy, gz = O.gradient(A)
    g2 = gx * gx + gy * gy + gz * gz
    qv = g2 / (g2 + 1e-10)
    expect = float(np.sum(qv * qv)) / np.prod([n - abs(c) for c in t])
    assert best == pytest.approx(expect, rel=1e-12)


def test_ramps_closed_form_with_rotation():
    """A = a (u_A . x), B = b (u_B . y): after B_hat = B o T the NGF direction
    is R^T u_B, so every valid shift scores (u_A . R^T u_B)^2 q_A q_B."""
    n = 13
    dims = (n, n, n)
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for _ in range(3)], indexing="ij")
    uA = np.array([1.0, 0.0, 0.0])
    uB = np.array([0.0, 0.6, 0.8])
    a, b = 2e-5, 5e-5
    A = a * (uA[0] * xx + uA[1] * yy + uA[2] * zz)
    B = b * (uB[0] * xx + uB[1] * yy + uB[2] * zz)
    MA = np.zeros(dims, np.uint8)
    MA[1:-1, 1:-1, 1:-1] = 1
    MB = np.zeros(dims, np.uint8)
    MB[3:-3, 3:-3, 3:-3] = 1
    q = synth.axis_angle_quaternion([0.3, 1.0, 0.2], 0.5)
    R = O.quat_to_rotmat(q)
    s, _ = O.score_map(A, MA, B, MB, q, eps=1e-5, gamma=0.5)
    fin = s[np.isfinite(s)]
    qa = a * a / (a * a + 1e-10)
    qb = b * b / (b * b + 1e-10)
    expect = (uA @ (R.T @ uB)) ** 2 * qa * qb
    wrong = (uA @ (R @ uB)) ** 2 * qa * qb
    assert abs(expect - wrong) > 1e-2
    assert fin.size > 10
    np.testing.assert_allclose(fin, expect, rtol=2e-7)


def test_generator_pair_recovers_truth_small():
    p = synth.config_pair(0)
    s, r, chi = O.align(p.A, p.MA, p.B, p.MB, p.quats)
    assert r == p.true_index
    assert chi == p.t_zyx


# ------------------------------------- rotated mask at fractional weights
def scalar_resample(B, MB, R, slack=1e-4):
    """B_hat and M_hat voxel by voxel from the Section 3.2 reading, written
    independently of the oracle: the sample point p = R (x - c) + c (FP32,
    in the order the reading fixes), the domain test against [0, n-1] with
    the slack, then trilinear interpolation in its hat-function form,
    f(p) = sum_k f[k] prod_i max(0, 1 - |p_i - k_i|) over the grid (FP64, at
    p clamped onto the box), with no base index or cell logic.  Returns the
    intensities, the interpolated mask m (FP64) and the domain flags."""
    nz, ny, nx = B.shape
    n = (nx, ny, nz)
    f32 = np.float32
    Rf = R.astype(f32)
    c = [f32((v - 1) / 2) for v in n]
    val = np.zeros(B.shape)
    mval = np.zeros(B.shape)
    inside = np.zeros(B.shape, dtype=bool)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                d = (f32(x) - c[0], f32(y) - c[1], f32(z) - c[2])
                p = []
                for i in range(3):
                    acc = f32(Rf[i, 0] * d[0])
                    acc = f32(acc + f32(Rf[i, 1] * d[1]))
                    acc = f32(acc + f32(Rf[i, 2] * d[2]))
                    p.append(float(f32(acc + c[i])))
                ok = all(-slack <= p[i] <= (n[i] - 1) + slack for i in range(3))
                inside[z, y, x] = ok
                pc = [min(max(p[i], 0.0), float(n[i] - 1)) for i in range(3)]
                hats = [[(k, max(0.0, 1.0 - abs(pc[i] - k))) for k in range(n[i])] for i in range(3)]
                hats = [[(k, w) for k, w in h if w > 0.0] for h in hats]
                v = m = 0.0
                for kz, wz in hats[2]:
                    for ky, wy in hats[1]:
                        for kx, wx in hats[0]:
                            v += wz * wy * wx * float(B[kz, ky, kx])
                            m += wz * wy * wx * float(MB[kz, ky, kx])
                val[z, y, x] = v if ok else 0.0
                mval[z, y, x] = m
    return val, mval, inside


def _check_resample_against_scalar(B, MB, q, require_exact_half=False):
    """The oracle's resample against the scalar definition: intensities to
    1e-12, and the mask decision [m >= 1/2] and domain test wherever the
    FP32 lerps cannot round across the half (|m - 1/2| > 1e-6); where m is
    exactly 1/2 the decision must be 'on'.  Returns (exact halves, skipped)."""
    R = O.quat_to_rotmat(q)
    Bh, Mh = O.resample(B, MB, q)
    val, m, inside = scalar_resample(B, MB, R)
    np.testing.assert_allclose(Bh, val, rtol=0, atol=1e-12)
    want = inside & (m >= 0.5)
    half = inside & (m == 0.5)
    decided = ~inside | (np.abs(m - 0.5) > 1e-6) | half
    assert np.array_equal(Mh.astype(bool)[decided], want[decided])
    if require_exact_half:
        assert decided.all()
    return int(half.sum()), int((~decided).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_resample_matches_scalar_definition_general_rotations(seed):
    """Non-axis rotations on tiny volumes: nearly every voxel has fractional
    weights on all three axes and many sample points leave the domain."""
    rng = np.random.default_rng(100 + seed)
    dims = [(5, 6, 4), (6, 6, 6), (4, 5, 6)][seed]
    B = rng.random(dims)
    MB = (rng.random(dims) < 0.5).astype(np.uint8)
    total_skipped = 0
    for q in synth.random_quaternions(rng, 4):
        _, skipped = _check_resample_against_scalar(B, MB, q)
        total_skipped += skipped
    assert total_skipped <= 2      # the check decides (almost) every voxel


def test_resample_mask_exactly_half_is_on():
    """A quarter turn about z on a 4 x 5 x 4 volume puts every sample point
    half-way between voxels in x and y (c_x = 1.5, c_y = 2), so the
    interpolated mask is the mean of four corners, exactly 1/2 wherever two
    are set (all FP32 lerps exact): those voxels must be in the mask.  Rows
    whose x sample lands at -0.5 or 3.5 fall outside the domain."""
    rng = np.random.default_rng(7)
    dims = (4, 5, 4)
    B = rng.random(dims)
    MB = (rng.random(dims) < 0.5).astype(np.uint8)
    q = synth.axis_angle_quaternion([0, 0, 1], np.pi / 2)
    halves, _ = _check_resample_against_scalar(B, MB, q, require_exact_half=True)
    assert halves >= 5
    R = O.quat_to_rotmat(q)
    _, _, inside = scalar_resample(B, MB, R)
    assert 0 < inside.sum() < inside.size


def test_resample_domain_slack_and_face_clamp():
    """A rotation of 7.5e-5 rad about z on a 5^3 volume moves the x sample
    points of the faces x = 0 and x = 4 by up to 1.5e-4: points within the
    1e-4 slack count as inside and sample the face itself; points beyond it
    are outside (B_hat = 0, mask 0)."""
    rng = np.random.default_rng(8)
    dims = (5, 5, 5)
    B = rng.random(dims) + 1.0
    MB = np.ones(dims, dtype=np.uint8)
    q = synth.axis_angle_quaternion([0, 0, 1], 7.5e-5)
    _check_resample_against_scalar(B, MB, q, require_exact_half=True)
    R = O.quat_to_rotmat(q)
    px, _, _ = O.sample_points_f32(R, dims)
    Bh, Mh = O.resample(B, MB, q)
    slack_pts = ((px < 0) & (px >= -1e-4)) | ((px > 4) & (px <= 4 + 1e-4))
    out_pts = (px < -1e-4) | (px > 4 + 1e-4)
    assert slack_pts.sum() >= 10 and out_pts.sum() >= 10
    assert np.all(Mh[slack_pts] == 1) and np.all(Mh[out_pts] == 0)
    assert np.all(Bh[out_pts] == 0.0)
    face = np.where(px[slack_pts] < 0, 0, 4)
    zs, ys, _ = np.nonzero(slack_pts)
    # at the slack points y is fractional, so compare with the face's own interpolation
    val, _, _ = scalar_resample(B, MB, R)
    np.testing.assert_allclose(Bh[slack_pts], val[slack_pts], rtol=0, atol=1e-12)
    assert len(face) == len(zs)


def test_best_of_map_tie_rule_by_scan():
    """The argmax tie rule (largest score, then the smallest (z, y, x) shift)
    against a plain lexicographic scan that keeps the first strictly larger
    value, on maps with planted equal maxima, -inf holes and an empty map."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        dims = tuple(int(v) for v in rng.integers(2, 5, size=3))
        shape = tuple(2 * n - 1 for n in dims)
        m = np.round(rng.random(shape), 1)          # many exact ties
        m[rng.random(shape) < 0.3] = -np.inf
        if trial == 0:
            m[:] = -np.inf
        best, chi = None, (0, 0, 0)
        for idx in itertools.product(*[range(s) for s in shape]):
            if np.isfinite(m[idx]) and (best is None or m[idx] > best):
                best, chi = float(m[idx]), tuple(i - (n - 1) for i, n in zip(idx, dims))
        got = O.best_of_map(m)
        if best is None:
            assert got[0] == -np.inf and got[1] == (0, 0, 0)
        else:
            assert got == (best, chi)


def test_align_tie_goes_to_smallest_rotation_index(monkeypatch):
    """Fig. 1's maximum over rotations: equal best scores go to the smallest
    rotation index (checked with a stand-in per-rotation scorer)."""
    monkeypatch.setattr(O, "score_rotations",
                        lambda *a, **k: (np.array([0.2, 0.7, 0.7, -np.inf]),
                                         np.array([[0, 0, 0], [1, 2, 3], [4, 5, 6], [0, 0, 0]])))
    assert O.align(None, None, None, None, [None] * 4) == (0.7, 1, (1, 2, 3))
    monkeypatch.setattr(O, "score_rotations",
                        lambda *a, **k: (np.full(3, -np.inf), np.zeros((3, 3), dtype=np.int64)))
    assert O.align(None, None, None, None, [None] * 3) == (-np.inf, -1, (0, 0, 0))


# ------------------------------------------------------------ mutations
def _pins_pass():
    """The pins re-run as plain functions; True if all of them pass."""
    checks = [
        test_direct_matches_brute_force_tiny,
        lambda: test_fft_form_equals_direct_all_shifts((6, 6, 6), 2),
        test_delta_fixes_shift_sign,
        test_ramps_closed_form_with_rotation,
        lambda: test_quarter_turn_resample_is_exact_permutation(2),
        test_integer_shift_at_identity_recovers_shift_and_closed_form,
        test_gradient_and_ngf_on_linear_ramp,
        lambda: test_resample_matches_scalar_definition_general_rotations(0),
        test_resample_mask_exactly_half_is_on,
        test_resample_domain_slack_and_face_clamp,
    ]
    try:
        for c in checks:
            c()
    except (AssertionError, IndexError):
        return False
    return True


def test_pins_pass_unmutated():
    assert _pins_pass()


@pytest.mark.parametrize("mutation", [
    "transpose_rotation", "drop_cross_weight", "flip_shift_sign",
    "eps_not_squared", "gradient_one_sided", "swap_xz_sample",
    "mask_strictly_above_half", "no_domain_slack", "no_clamp_onto_box", "lerp_weights_reversed",
])
def test_planted_mistakes_are_caught(mutation, monkeypatch):
    if mutation == "transpose_rotation":
        orig = O.quat_to_rotmat
        monkeypatch.setattr(O, "quat_to_rotmat", lambda q: orig(q).T.copy())
    elif mutation == "drop_cross_weight":
        monkeypatch.setattr(O, "CHANNEL_WEIGHTS", (1.0,) * 6)
    elif mutation == "flip_shift_sign":
        orig_g = O._gather_shifts
        monkeypatch.setattr(O, "_gather_shifts",
                            lambda c, dims, pad: orig_g(np.flip(np.roll(c, -1, axis=(0, 1, 2)),
                                                                axis=(0, 1, 2)), dims, pad))
    elif mutation == "eps_not_squared":
        def ngf_bad(V, eps):
            gx, gy, gz = O.gradient(V)
            inv = 1.0 / np.sqrt(gx * gx + gy * gy + gz * gz + float(eps))
            return gx * inv, gy * inv, gz * inv
        monkeypatch.setattr(O, "ngf", ngf_bad)
    elif mutation == "gradient_one_sided":
        def grad_bad(V):
            V = np.asarray(V, dtype=float)
            out = []
            for axis in (2, 1, 0):
                n = V.shape[axis]
                up = np.take(V, np.minimum(np.arange(n) + 1, n - 1), axis=axis)
                out.append(up - V)
            return tuple(out)
        monkeypatch.setattr(O, "gradient", grad_bad)
    elif mutation == "swap_xz_sample":
        orig_s = O.sample_points_f32
        monkeypatch.setattr(O, "sample_points_f32",
                            lambda R, dims: tuple(reversed(orig_s(R, dims))))
    elif mutation == "mask_strictly_above_half":
        monkeypatch.setattr(O, "_mask_on", lambda m: m > np.float32(0.5))
    elif mutation == "no_domain_slack":
        monkeypatch.setattr(O, "DOMAIN_SLACK", 0.0)
    elif mutation == "no_clamp_onto_box":
        def axis_bad(p, n):
            slack = np.float32(O.DOMAIN_SLACK)
            inside = (p >= -slack) & (p <= np.float32(n - 1) + slack)
            i0 = np.minimum(np.floor(p).astype(np.int64), max(n - 2, 0))
            t = (p - i0.astype(np.float32)).astype(np.float32)
            return inside, i0, t
        monkeypatch.setattr(O, "_axis_setup", axis_bad)
    elif mutation == "lerp_weights_reversed":
        monkeypatch.setattr(O, "_lerp", lambda a, b, t: (b + t * (a - b)).astype(np.float32))
    assert not _pins_pass(), f"mutation {mutation} went unnoticed"


# ------------------------------------------------------------ Eq. 3 (US-NGF)
def brute_us(A, MA, B, MB, eps, gamma):
    """Eq. 1, 3 and 5 with scalar loops only."""
    nz, ny, nx = A.shape

    def nvec(V, z, y, x):
        def at(zz, yy, xx):
            return V[min(max(zz, 0), nz - 1), min(max(yy, 0), ny - 1), min(max(xx, 0), nx - 1)]
        g = ((at(z, y, x + 1) - at(z, y, x - 1)) / 2, (at(z, y + 1, x) - at(z, y - 1, x)) / 2,
             (at(z + 1, y, x) - at(z - 1, y, x)) / 2)
        den = math.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2 + eps ** 2)
        return [v / den for v in g]

    thr = max(1, math.ceil(gamma * min(int(MA.sum()), int(MB.sum()))))
    out = {}
    for chi in itertools.product(*[range(-(n - 1), n) for n in A.shape]):
        num, N = 0.0, 0
        for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
            zb, yb, xb = z + chi[0], y + chi[1], x + chi[2]
            if 0 <= zb < nz and 0 <= yb < ny and 0 <= xb < nx and MA[z, y, x] and MB[zb, yb, xb]:
                a, b = nvec(A, z, y, x), nvec(B, zb, yb, xb)
                num += a[0] * b[0] + a[1] * b[1] + a[2] * b[2]
                N += 1
        out[chi] = num / N if N >= thr else -np.inf
    return out


def test_unsquared_direct_matches_brute_force_tiny():
    A, MA, B, MB = rand_case(12, (3, 3, 4))
    s, _ = O.csngf_direct(A, MA, B, MB, 0.05, 0.5, measure="unsquared")
    for chi, v in brute_us(A, MA, B, MB, 0.05, 0.5).items():
        idx = tuple(c + n - 1 for c, n in zip(chi, A.shape))
        if np.isfinite(v):
            assert s[idx] == pytest.approx(v, rel=1e-12, abs=1e-14)
        else:
            assert not np.isfinite(s[idx])


def test_unsquared_fft_equals_direct():
    A, MA, B, MB = rand_case(13, (6, 7, 5))
    s_d, _ = O.csngf_direct(A, MA, B, MB, 1e-3, 0.5, measure="unsquared")
    s_f, _ = O.csngf_fft(A, MA, B, MB, 1e-3, 0.5, measure="unsquared")
    fin = np.isfinite(s_d)
    assert np.array_equal(fin, np.isfinite(s_f))
    np.testing.assert_allclose(s_f[fin], s_d[fin], rtol=1e-10, atol=1e-12)


def test_unsquared_is_sign_sensitive_and_bounded():
    A, MA, B, MB = rand_case(14, (6, 6, 6))
    s1, _ = O.csngf_fft(A, MA, B, MB, 1e-3, 0.5, measure="unsquared")
    s2, _ = O.csngf_fft(A, MA, -B, MB, 1e-3, 0.5, measure="unsquared")
    fin = np.isfinite(s1)
    np.testing.assert_allclose(s2[fin], -s1[fin], rtol=1e-12, atol=1e-14)
    assert s1[fin].min() >= -1 - 1e-12 and s1[fin].max() <= 1 + 1e-12


def test_unsquared_ramps_closed_form_with_rotation():
    n = 13
    zz, yy, xx = np.meshgrid(*[np.arange(n, dtype=float) for _ in range(3)], indexing="ij")
    uA, uB = np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.6, 0.8])
    a, b = 2e-5, 5e-5
    A = a * (uA[0] * xx + uA[1] * yy + uA[2] * zz)
    B = b * (uB[0] * xx + uB[1] * yy + uB[2] * zz)
    MA = np.zeros((n, n, n), np.uint8)
    MA[1:-1, 1:-1, 1:-1] = 1
    MB = np.zeros((n, n, n), np.uint8)
    MB[3:-3, 3:-3, 3:-3] = 1
    q = synth.axis_angle_quaternion([0.3, 1.0, 0.2], 0.5)
    R = O.quat_to_rotmat(q)
    s, _ = O.score_map(A, MA, B, MB, q, eps=1e-5, measure="unsquared")
    fin = s[np.isfinite(s)]
    expect = (uA @ (R.T @ uB)) * math.sqrt(a * a / (a * a + 1e-10)) * math.sqrt(b * b / (b * b + 1e-10))
    np.testing.assert_allclose(fin, expect, rtol=2e-7)


# --------------------------------------------- slab bound used to prune shifts
def slab_bound(MA, MB, axis):
    """U(c) = sum_i min(a_i, b_{i+c}) over the slabs along one axis."""
    others = tuple(a for a in range(3) if a != axis)
    a = MA.sum(axis=others).astype(np.int64)
    b = MB.sum(axis=others).astype(np.int64)
    n = len(a)
    return {c: sum(min(a[i], b[i + c]) for i in range(max(0, -c), min(n, n - c))) for c in range(-(n - 1), n)}


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_slab_bound_never_below_overlap(seed):
    """N(chi) <= min over axes of the slab bound, so a shift whose bound is
    below the overlap threshold is invalid (exact pruning of the inverse)."""
    rng = np.random.default_rng(seed)
    dims = (7, 8, 6)
    MA = (rng.random(dims) < 0.5).astype(np.uint8)
    MB = (rng.random(dims) < 0.4).astype(np.uint8)
    _, N = O.csngf_direct(rng.random(dims), MA, rng.random(dims), MB, 1e-3, 0.5)
    bounds = [slab_bound(MA, MB, ax) for ax in range(3)]
    for idx in itertools.product(*[range(2 * n - 1) for n in dims]):
        chi = [i - (n - 1) for i, n in zip(idx, dims)]
        assert N[idx] <= min(bounds[ax][chi[ax]] for ax in range(3))


# --------------------------------------- bound-limited FFT length (alias-free)
@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_shorter_circular_length_is_exact_on_a_shift_range(seed):
    """A length-P circular correlation holds at slot chi mod P the sum of the
    linear one over chi + kP.  For shifts in [lo, hi] with P >= n + max(-lo,
    hi), every chi + kP (k != 0) leaves the linear support [-(n-1), n-1], so
    the slots equal the linear correlation there (checked against the direct
    sum); one slot shorter, a boundary shift picks up an alias (positive
    inputs make every linear value nonzero)."""
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(5, 9, size=3))
    a = rng.random(dims) + 0.1
    b = rng.random(dims) + 0.1
    lo = [int(rng.integers(-(n - 1), 1)) for n in dims]
    hi = [int(rng.integers(0, n)) for n in dims]
    P = [n + max(-l, h) for n, l, h in zip(dims, lo, hi)]
    box = tuple(slice(l + n - 1, h + n) for l, h, n in zip(lo, hi, dims))
    ref = np.zeros(tuple(2 * n - 1 for n in dims))
    for chi in itertools.product(*[range(-(n - 1), n) for n in dims]):
        sa, sb = O._shift_slices(chi, dims, dims)
        ref[tuple(c + n - 1 for c, n in zip(chi, dims))] = float((a[sa] * b[sb]).sum())
    got = O.correlate_fft(a, b, tuple(P))
    np.testing.assert_allclose(got[box], ref[box], rtol=1e-12, atol=1e-12)
    for ax in range(3):
        if P[ax] - 1 < dims[ax]:
            continue
        short = list(P)
        short[ax] -= 1
        bad = O.correlate_fft(a, b, tuple(short))
        assert np.max(np.abs(bad[box] - ref[box])) > 1e-3

