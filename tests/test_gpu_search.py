"""The pyramid random-search driver (Section 3.2) against its FP64 reference,
and recovery of a known transform."""
import math

import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from oracle import search_oracle as S
from paper_2110_10156_gb300 import synth

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


def test_search_matches_reference_driver(cs):
    p = synth.small_pair(301, (24, 22, 26), masks="threshold", max_shift=2)
    schedule = [(1.0, 2, 40.0, 24, 1), (0.0, 1, 8.0, 10, 4)]
    g = cs.global_align(dev(p.A), dev(p.MA), dev(p.B), dev(p.MB), schedule=schedule, seed=99)
    score, euler, shift, level_best, _ = S.global_align(p.A, p.MA, p.B, p.MB, schedule, 99)
    assert g["rotations_scored"] == 25 + 14
    for a, b in zip(g["level_best"], level_best):
        assert a == pytest.approx(b, rel=1e-4, abs=1e-5)
    assert g["score"] == pytest.approx(score, rel=1e-4)
    np.testing.assert_allclose(g["euler_deg"], euler, rtol=0, atol=1e-9)
    assert g["shift"] == shift


def corner_error(q_found, chi_found, q_true, t_true, dims):
    """Mean distance over the 8 corners between where the found and the true
    transform send each corner of A into B's frame (the d_E of Section 5.1)."""
    n = np.array(dims[::-1], dtype=float)              # (x, y, z)
    c = (n - 1) / 2
    Rf, Rt = O.quat_to_rotmat(q_found), O.quat_to_rotmat(q_true)
    cf = np.array(chi_found[::-1], dtype=float)
    ct = np.array(t_true[::-1], dtype=float)
    err = []
    for corner in np.array(np.meshgrid([0, 1], [0, 1], [0, 1])).reshape(3, -1).T:
        x = corner * (n - 1)
        yf = Rf @ (x + cf - c) + c
        yt = Rt @ (x + ct - c) + c
        err.append(np.linalg.norm(yf - yt))
    return float(np.mean(err))


def test_search_recovers_known_transform(cs):
    p = synth.make_pair(77, (48, 48, 48), 14, 3.0, 12.0, 25.0, 4, 2, masks="threshold", sigma=1.0)
    schedule = [(2.0, 4, 180.0, 600, 1), (1.0, 2, 20.0, 200, 6), (0.0, 1, 4.0, 40, 2)]
    g = cs.global_align(dev(p.A), dev(p.MA), dev(p.B), dev(p.MB), schedule=schedule, seed=5)
    d_e = corner_error(g["quat"], g["shift"], p.q_true, p.t_zyx, p.A.shape)
    assert d_e < 5.0, (g, p.q_true, p.t_zyx, d_e)
