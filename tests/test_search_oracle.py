"""Pins for the search driver's reference: SplitMix64 against its published
reference outputs, Euler angles against scipy, the pyramid levels against
scipy's Gaussian filter definition."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import search_oracle as S


def test_splitmix64_matches_published_sequence():
    # first outputs for seed 1234567 from the reference C implementation
    # (Vigna, splitmix64.c)
    rng = S.SplitMix64(1234567)
    got = [rng.next() for _ in range(5)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_in_unit_interval():
    rng = S.SplitMix64(7)
    u = np.array([rng.uniform() for _ in range(2000)])
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.03


def test_euler_intrinsic_xyz_matches_scipy():
    rng = np.random.default_rng(1)
    for _ in range(10):
        e = rng.uniform(-180, 180, 3)
        q = S.euler_to_quat(e)
        R = Rotation.from_euler("XYZ", e, degrees=True).as_matrix()    # intrinsic x, y', z''
        from oracle import cs_ngf_oracle as O
        np.testing.assert_allclose(O.quat_to_rotmat(q), R, atol=1e-12)


def test_level_volume_definition():
    rng = np.random.default_rng(2)
    V = rng.random((9, 10, 11))
    M = (rng.random((9, 10, 11)) > 0.5).astype(np.uint8)
    L, LM = S.level_volume(V, M, 1.5, 2)
    from scipy import ndimage
    ref = ndimage.gaussian_filter(V, 1.5, mode="nearest", truncate=4.0)[::2, ::2, ::2]
    np.testing.assert_allclose(L, ref, rtol=1e-12, atol=1e-14)
    assert L.shape == (5, 5, 6) and np.array_equal(LM, M[::2, ::2, ::2])


# ---- the search driver's bookkeeping against Section 3.2 ----------------------
def _tiny_pair():
    from paper_2110_10156_gb300 import synth
    return synth.small_pair(17, (10, 11, 12), n_rot=1, masks="full")


def test_start_point_alone_scores_as_the_scoring_oracle():
    """With no random rotations a level scores only its starting points: the
    result is the scoring oracle's best (score, shift) at the start rotation."""
    from oracle import cs_ngf_oracle as O
    p = _tiny_pair()
    start = (7.0, -12.0, 25.0)
    score, euler, shift, level_best, cands = S.global_align(
        p.A, p.MA, p.B, p.MB, [(0.0, 1, 0.0, 0, 1)], seed=3, start=start)
    s, c = O.score_rotations(p.A, p.MA, p.B, p.MB, [S.euler_to_quat(start)])
    assert euler == start and score == s[0] and shift == tuple(int(v) for v in c[0])
    assert level_best == [score] and cands[0][0] == [start]


def test_levels_carry_their_best_candidates_and_rescore_them():
    """Level k's starting points are the p_{k+1} best candidates of level k
    (stable order on equal scores), each scored again at level k+1 before its
    random rotations; random rotations lie within +-u of a starting point on
    every Euler angle."""
    p = _tiny_pair()
    schedule = [(0.0, 1, 40.0, 8, 1), (0.0, 1, 10.0, 5, 3), (0.0, 1, 0.0, 0, 2)]
    _, _, _, level_best, cands = S.global_align(p.A, p.MA, p.B, p.MB, schedule, seed=11)
    assert len(cands) == 3
    for k in range(2):
        cand, scores, _ = cands[k]
        keep = schedule[k + 1][4]
        order = sorted(range(len(cand)), key=lambda i: (-scores[i], i))
        best = [cand[i] for i in order[:keep]]
        nxt = cands[k + 1][0]
        assert nxt[:keep] == best                         # re-evaluated first
        assert level_best[k] == max(scores)
        u = schedule[k + 1][2]
        for e in nxt[keep:]:                              # a_{k+1} random rotations
            assert any(all(abs(e[a] - b[a]) <= u for a in range(3)) for b in best)
        assert len(nxt) == keep + schedule[k + 1][3]
    # level 0 starts from the given point, with a_0 random rotations around it
    assert cands[0][0][0] == (0.0, 0.0, 0.0) and len(cands[0][0]) == 1 + 8


def test_downsampled_level_reports_full_resolution_shift():
    """A level that keeps every d-th voxel finds shifts in its own voxels; the
    driver reports them in full-resolution voxels (times d)."""
    from oracle import cs_ngf_oracle as O
    p = _tiny_pair()
    _, _, shift, _, cands = S.global_align(p.A, p.MA, p.B, p.MB, [(0.0, 2, 0.0, 0, 1)], seed=5)
    level_shift = cands[0][2][0]
    assert shift == tuple(2 * int(v) for v in level_shift)
    A2, M2 = S.level_volume(p.A, p.MA, 0.0, 2)
    B2, MB2 = S.level_volume(p.B, p.MB, 0.0, 2)
    _, c = O.score_rotations(A2, M2, B2, MB2, [S.euler_to_quat((0.0, 0.0, 0.0))])
    assert tuple(int(v) for v in c[0]) == tuple(int(v) for v in level_shift)
