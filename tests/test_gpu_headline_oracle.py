"""The 150^3 workload with all 1000 rotations against the FP64 oracle's
per-rotation results (Section 3.2: the argmax over the shifts of each
rotation, then the maximum over rotations, Fig. 1), in the launch
configuration the bench times (automatic batch, bound-limited padding).

tests/golden/oracle_headline_150cubed.json holds, for every rotation, the
oracle's best score s1 and shift at the full linear length (320^3), the best
score s2 outside the 3x3x3 neighbourhood of that shift and the largest |score|,
written by tests/golden/make_oracle_headline.py (which calls only the oracle).

The argmax rule: where s1 - s2 > 2 tau s1 the GPU returns exactly the
oracle's shift; elsewhere the oracle's own score at the GPU's shift (its
direct Eq. 5 sum) is within tau s1 of s1.  The GPU's score is within tau of
the oracle's score at that shift (scores lie in [0, 1])."""
import json
import os

import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_headline_150cubed.json")


@pytest.fixture(scope="module")
def cs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    return cs_ngf


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


@pytest.fixture(scope="module")
def pair():
    return synth.config_pair(1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oracle_at(p, r, chi):
    """The oracle's direct Eq. 5 sum for rotation r at one shift."""
    Bh, Mh = O.resample(p.B, p.MB, p.quats[r])
    m, _ = O.csngf_direct(p.A, p.MA, Bh, Mh, 1e-5, 0.5, chis=[tuple(int(v) for v in chi)])
    return float(m[tuple(int(c) + n - 1 for c, n in zip(chi, p.A.shape))])


def score_all(cs, p, precision, **kw):
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), precision=precision, **kw)
    B, MB = dev(p.B), dev(p.MB)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(B, MB, p.quats)]
    align = f.align(B, MB, p.quats)
    f.release()
    return sc, sh, align


def check_global(golden, align, tau):
    s1 = np.array(golden["s1"])
    b = golden["best_rotation"]
    others = np.delete(s1, b)
    runner = max(float(others.max()), float(golden["s2"][b]))
    assert s1[b] - runner > 2 * tau * s1[b]            # this workload's maximum is unambiguous
    score, ri, chi = align
    assert ri == b and list(chi) == golden["shift"][b], (ri, chi)
    assert abs(score - s1[b]) <= tau


def test_fp32_every_rotation_against_the_oracle(cs, golden, pair):
    tau = 1e-4
    p = pair
    assert golden["rotations"] == len(p.quats) and golden["true_index"] == p.true_index
    sc, sh, align = score_all(cs, p, "fp32")
    s1, s2 = np.array(golden["s1"]), np.array(golden["s2"])
    near = []
    for r in range(len(p.quats)):
        assert np.isfinite(sc[r])
        if s1[r] - s2[r] > 2 * tau * s1[r]:
            assert list(sh[r]) == golden["shift"][r], (r, sh[r], golden["shift"][r])
            assert abs(float(sc[r]) - s1[r]) <= tau, (r, sc[r], s1[r])
        else:
            near.append(r)
    assert len(near) <= 30
    for r in near:                                     # near-ties: the oracle's own score there
        o = oracle_at(p, r, sh[r])
        assert abs(float(sc[r]) - o) <= tau, (r, sc[r], o)
        assert o >= s1[r] - tau * s1[r], (r, o, s1[r])
    check_global(golden, align, tau)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_reduced_precision_every_rotation_against_the_oracle(cs, golden, pair, precision):
    """tau = 1e-2: nearly every rotation is a near-tie at this tolerance, so
    each GPU best score must lie within 2 tau of the oracle's best (it is
    within tau of the oracle's score at a shift scoring at least s1 - tau s1),
    the exact shift where the gap rule asks for it, the full rule on a sample
    of rotations by the oracle's direct sum, and the global maximum exactly."""
    tau = 1e-2
    p = pair
    sc, sh, align = score_all(cs, p, precision)
    s1, s2 = np.array(golden["s1"]), np.array(golden["s2"])
    assert np.all(np.abs(sc.astype(np.float64) - s1) <= 2 * tau)
    for r in range(len(p.quats)):
        if s1[r] - s2[r] > 2 * tau * s1[r]:
            assert list(sh[r]) == golden["shift"][r], (r, sh[r], golden["shift"][r])
    rng = np.random.default_rng(7)
    for r in [golden["best_rotation"]] + [int(i) for i in rng.choice(len(p.quats), 4, replace=False)]:
        o = oracle_at(p, r, sh[r])
        assert abs(float(sc[r]) - o) <= tau, (r, sc[r], o)
        assert o >= s1[r] - tau * s1[r], (r, o, s1[r])
    check_global(golden, align, tau)
