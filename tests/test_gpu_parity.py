"""CUDA path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth
from tests.parity_util import TAU_FP32, check_best_against_map, check_maps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    return cs_ngf


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rand_quat(seed):
    return synth.random_quaternions(np.random.default_rng(seed), 1)[0]


IDENTITY = np.array([1.0, 0.0, 0.0, 0.0])


# ------------------------------------------------------------ Section 3.2 resample
@pytest.mark.parametrize("dims", [(12, 10, 14), (21, 17, 9), (32, 32, 32)])
def test_resample_matches_oracle(cs, dims):
    p = synth.small_pair(5, dims, masks="threshold")
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    quats = [IDENTITY, rand_quat(1), rand_quat(2),
             synth.axis_angle_quaternion([0, 0, 1], np.pi / 2)]
    for q in quats:
        Bh, Mh = f.resample(dev(p.B), dev(p.MB), q)
        oB, oM = O.resample(p.B, p.MB, q)
        np.testing.assert_array_equal(Mh.cpu().numpy(), oM)           # integer decision: exact
        np.testing.assert_allclose(Bh.cpu().numpy(), oB, rtol=0, atol=2e-6 * max(1.0, np.abs(p.B).max()))
    f.release()


# ------------------------------------------------------------ Eq. 5 score maps
MAP_CASES = [
    ((8, 8, 8), (16, 16, 16)),
    ((12, 10, 14), None),                   # 32^3
    ((20, 17, 23), None),                   # 64^3
    ((33, 40, 30), None),                   # 128, 128, 64
    ((9, 8, 10), (400, 32, 160)),
    ((10, 12, 9), (200, 512, 256)),
    ((7, 9, 8), (32, 400, 512)),
    ((16, 15, 14), (320, 320, 320)),
    ((9, 10, 8), (192, 216, 192)),          # radix-3 lengths, half-length inputs
    ((11, 8, 10), (216, 192, 216)),
    ((9, 8, 10), (360, 32, 360)),           # 18 x 20
]


def pad_mode_for(pad):
    """Requested lengths are tested as given (full padding); automatic ones
    with the default bound-limited padding."""
    return "bound" if pad is None else "full"


@pytest.mark.parametrize("dims,pad", MAP_CASES)
def test_score_map_matches_oracle(cs, dims, pad):
    p = synth.small_pair(11 + sum(dims), dims, masks="threshold")
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad=pad, pad_mode=pad_mode_for(pad))
    for q in (IDENTITY, p.q_true, rand_quat(sum(dims))):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        if pad is not None:
            assert f.pad == tuple(pad)
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad)
        check_maps(omap, gmap)
    f.release()


def test_score_map_full_masks(cs):
    p = synth.small_pair(3, (14, 13, 12), masks="full")
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    for q in (IDENTITY, rand_quat(9)):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_maps(omap, gmap)


# ------------------------------------------------------------ argmax per rotation
def test_score_rotations_small_workload_32(cs):
    p = synth.config_pair(0)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    sc, sh = f.score_rotations(dev(p.B), dev(p.MB), p.quats)
    sc, sh = sc.cpu().numpy(), sh.cpu().numpy()
    kinds = []
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        kinds.append(check_best_against_map(omap, sc[r], sh[r]))
    assert kinds.count("exact") >= 6
    score, ri, chi = f.align(dev(p.B), dev(p.MB), p.quats)
    assert ri == p.true_index and chi == p.t_zyx
    assert score == pytest.approx(float(sc[ri]))


def test_batches_do_not_change_results(cs):
    p = synth.small_pair(21, (18, 16, 20), n_rot=11)
    quats = np.concatenate([p.quats, synth.random_quaternions(np.random.default_rng(4), 6)])
    f1 = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=3)
    f2 = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=17)
    # odd batches round down to even: masks of rotations 2k, 2k+1 share a transform
    assert (f1.batch, f2.batch) == (2, 16)
    a1 = [t.cpu().numpy() for t in f1.score_rotations(dev(p.B), dev(p.MB), quats)]
    a2 = [t.cpu().numpy() for t in f2.score_rotations(dev(p.B), dev(p.MB), quats)]
    np.testing.assert_array_equal(a1[0], a2[0])
    np.testing.assert_array_equal(a1[1], a2[1])


def test_host_entry_point_equals_device_entry_point(cs):
    p = synth.small_pair(31, (16, 16, 16), n_rot=5)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    d_sc, d_sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    h_sc, h_sh = f.score_rotations_host(p.B, p.MB, p.quats)
    np.testing.assert_array_equal(d_sc, h_sc)
    np.testing.assert_array_equal(d_sh, h_sh)


# ------------------------------------------------------------ invariants, edge cases
def test_negated_intensity_is_bit_identical(cs):
    p = synth.small_pair(41, (20, 18, 16), n_rot=6)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    a = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    b = [t.cpu().numpy() for t in f.score_rotations(dev(-p.B), dev(p.MB), p.quats)]
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def _permute(V, R):
    n = V.shape[0]
    idx = np.arange(n)
    zb, yb, xb = np.meshgrid(idx, idx, idx, indexing="ij")
    d2 = np.stack([2 * xb - (n - 1), 2 * yb - (n - 1), 2 * zb - (n - 1)], axis=-1)
    s2 = d2 @ R + (n - 1)                      # rows: R^T d
    xa, ya, za = s2[..., 0] // 2, s2[..., 1] // 2, s2[..., 2] // 2
    return V[za, ya, xa]


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_quarter_turn_equals_identity_map(cs, axis):
    p = synth.small_pair(51, (15, 15, 15))
    q = synth.axis_angle_quaternion(np.eye(3)[axis], np.pi / 2)
    R = np.rint(O.quat_to_rotmat(q)).astype(int)
    B = _permute(p.A, R).astype(np.float32)
    MB = _permute(p.MA, R).astype(np.uint8)
    # one FFT geometry for both maps (bound-limited lengths follow each call's masks)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad_mode="full")
    m_rot = f.score_map(dev(B), dev(MB), q).cpu().numpy()
    m_id = f.score_map(dev(p.A), dev(p.MA), IDENTITY).cpu().numpy()
    np.testing.assert_array_equal(m_rot, m_id)
    s, ri, chi = f.align(dev(B), dev(MB), [IDENTITY, q])
    assert ri == 1 and chi == (0, 0, 0)


def test_empty_mask_gives_no_valid_shift(cs):
    p = synth.small_pair(61, (10, 10, 10), n_rot=3)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    zero = np.zeros_like(p.MB)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(zero), p.quats)]
    assert np.all(np.isneginf(sc)) and np.all(sh == 0)
    s, ri, chi = f.align(dev(p.B), dev(zero), p.quats)
    assert ri == -1 and np.isneginf(s)


def test_rotation_out_of_domain_mask(cs):
    """A mask that a rotation moves entirely out of the domain has no valid shift
    for that rotation only."""
    n = 12
    p = synth.small_pair(71, (n, n, n), n_rot=2)
    MB = np.zeros((n, n, n), np.uint8)
    MB[0, 0, :] = 1                                  # a corner edge line
    q = synth.axis_angle_quaternion([1, 1, 0], np.pi / 4)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    sc, _ = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(MB), [IDENTITY, q])]
    for r, qq in enumerate([IDENTITY, q]):
        omap, _ = O.score_map(p.A, p.MA, p.B, MB, qq)
        assert np.isfinite(sc[r]) == bool(np.isfinite(omap).any())


def test_bad_arguments_raise(cs):
    p = synth.small_pair(81, (8, 8, 8), n_rot=2)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    with pytest.raises(cs.CsNgfError) as e:
        f.score_rotations(dev(p.B), dev(p.MB), [[2.0, 0, 0, 0]])
    assert e.value.status == cs.EINVAL
    with pytest.raises(cs.CsNgfError):
        f.score_rotations(dev(p.B), dev(p.MB), np.zeros((0, 4)))


def test_minimum_sizes(cs):
    rng = np.random.default_rng(3)
    for dims in [(2, 2, 2), (2, 5, 3)]:
        A = rng.random(dims).astype(np.float32)
        B = rng.random(dims).astype(np.float32)
        M = np.ones(dims, np.uint8)
        f = cs.prepare_fixed(dev(A), dev(M), eps=1e-3)
        gmap = f.score_map(dev(B), dev(M), IDENTITY).cpu().numpy()
        omap, _ = O.score_map(A, M, B, M, IDENTITY, eps=1e-3)
        check_maps(omap, gmap)


def test_graph_replay_matches_direct_launches(cs):
    """Full batches replay one captured CUDA graph; with profiling on every
    kernel is launched directly.  Both give identical results, also after the
    fixed volume is replaced by one with a different mask sum."""
    p = synth.small_pair(91, (14, 16, 15), n_rot=9)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4)
    a = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    f.set_profiling(True)
    b = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    f.stage_times()
    f.set_profiling(False)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    MA2 = p.MA.copy()
    MA2[: p.MA.shape[0] // 2] = 0
    f.update_fixed(dev(p.A), dev(MA2))
    c = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    g = cs.prepare_fixed(dev(p.A), dev(MA2), batch=4)
    d = [t.cpu().numpy() for t in g.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    np.testing.assert_array_equal(c[0], d[0])
    np.testing.assert_array_equal(c[1], d[1])


# ------------------------------------------------------------ Eq. 3 (US-NGF)
@pytest.mark.parametrize("dims,pad", [((12, 10, 14), None), ((20, 17, 23), None), ((9, 8, 10), (400, 32, 160))])
def test_unsquared_measure_matches_oracle(cs, dims, pad):
    p = synth.small_pair(211 + sum(dims), dims, masks="threshold")
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad=pad, measure="unsquared", pad_mode=pad_mode_for(pad))
    for q in (IDENTITY, p.q_true, rand_quat(7)):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad, measure="unsquared")
        check_maps(omap, gmap)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad, measure="unsquared")
        check_best_against_map(omap, sc[r], sh[r])


def test_unsquared_measure_flips_sign_under_negation(cs):
    p = synth.small_pair(223, (16, 14, 12))
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), measure="unsquared")
    m1 = f.score_map(dev(p.B), dev(p.MB), IDENTITY).cpu().numpy()
    m2 = f.score_map(dev(-p.B), dev(p.MB), IDENTITY).cpu().numpy()
    fin = np.isfinite(m1)
    np.testing.assert_array_equal(fin, np.isfinite(m2))
    np.testing.assert_allclose(m2[fin], -m1[fin], rtol=0, atol=1e-6)


# ------------------------------------------------------------ BF16 storage form
TAU_BF16 = 1e-2


@pytest.mark.parametrize("dims,pad", [((12, 10, 14), None), ((20, 17, 23), None), ((16, 15, 14), (320, 320, 320))])
def test_bf16_form_within_reduced_precision_tolerance(cs, dims, pad):
    p = synth.small_pair(331 + sum(dims), dims, masks="threshold")
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad=pad, precision="bf16", pad_mode=pad_mode_for(pad))
    worst = 0.0
    for q in (IDENTITY, p.q_true, rand_quat(3)):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad)
        worst = max(worst, check_maps(omap, gmap, tau=TAU_BF16))
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad)
        check_best_against_map(omap, sc[r], sh[r], tau=TAU_BF16)
    assert worst > 0.0          # the reduced-precision path really differs from FP32 arithmetic


# ------------------------------------------------------------ FP16 storage form
@pytest.mark.parametrize("dims,pad", [((12, 10, 14), None), ((20, 17, 23), None), ((16, 15, 14), (320, 320, 320))])
def test_fp16_form_within_reduced_precision_tolerance(cs, dims, pad):
    """FP16 intermediates (per-field power-of-two scales): within the reduced
    precision budget of the FP64 oracle, and closer to it than BF16."""
    p = synth.small_pair(331 + sum(dims), dims, masks="threshold")
    errs = {}
    for prec in ("fp16", "bf16"):
        f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad=pad, precision=prec, pad_mode=pad_mode_for(pad))
        worst = 0.0
        for q in (IDENTITY, p.q_true, rand_quat(3)):
            gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
            omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad)
            worst = max(worst, check_maps(omap, gmap, tau=TAU_BF16))
        if prec == "fp16":
            sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
            for r, q in enumerate(p.quats):
                omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad)
                check_best_against_map(omap, sc[r], sh[r], tau=TAU_BF16)
        errs[prec] = worst
        f.release()
    assert 0.0 < errs["fp16"] < errs["bf16"]


def test_fp16_form_scales_wide_planes(cs):
    """Planes of 190 x 180 voxels: after the y pass a channel field can reach
    about 34,000 per unit of NGF product, past half of FP16's range, so the
    fields are stored at half scale.  The maps stay within the budget."""
    p = synth.small_pair(707, (6, 190, 180), masks="threshold", n_rot=2)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), precision="fp16")
    g = cs.prepare_fixed(dev(p.A), dev(p.MA))
    for q in (IDENTITY, p.q_true):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_maps(omap, gmap, tau=TAU_BF16)
        fmap = g.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        fin = np.isfinite(fmap)
        assert np.max(np.abs(gmap[fin] - fmap[fin])) <= 2e-3 * np.max(np.abs(fmap[fin]))
