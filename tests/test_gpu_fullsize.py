"""Full-size parity: the 150^3 workload with 1000 rotations and the 256^3
workload with 5000 rotations, scored in
the same launch configuration the bench times (automatic batch), checked
against the FP64 oracle on sampled rotations and by properties on all."""
import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth
from tests.parity_util import (check_best_against_map, check_best_at_sampled_shifts, check_maps,
                               face_neighbours)

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


@pytest.fixture(scope="module")
def pair150():
    return synth.config_pair(1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def oracle150(pair150):
    """The oracle's full maps (FFT form at 320^3) for q_true and two sampled rotations."""
    p = pair150
    rng = np.random.default_rng(99)
    sample = [p.true_index] + [int(i) for i in rng.choice(len(p.quats), 2, replace=False)]
    return {r: O.score_map(p.A, p.MA, p.B, p.MB, p.quats[r], pad=(320, 320, 320))[0] for r in sample}


@pytest.mark.parametrize("precision,tau,pad_mode", [("fp32", 1e-4, "bound"), ("bf16", 1e-2, "bound"),
                                                    ("fp16", 1e-2, "bound"), ("fp32", 1e-4, "full")])
def test_150_cubed_1000_rotations(cs, pair150, oracle150, precision, tau, pad_mode):
    p = pair150
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), precision=precision, pad_mode=pad_mode)
    assert f.max_pad == (320, 320, 320)
    assert f.sum_mask_a == int(p.MA.sum())
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    if pad_mode == "full":
        assert f.pad == (320, 320, 320)
    else:                   # every shift the overlap bound admits lies within about +-60
        assert all(v < 320 for v in f.pad), f.pad
    R = len(p.quats)
    assert sc.shape == (R,) and sh.shape == (R, 3)
    # properties at any size: scores are averages of values in [0, 1]; shifts in range
    fin = np.isfinite(sc)
    assert fin.all()
    assert sc.min() >= -1e-6 and sc.max() <= 1 + 1e-6
    assert np.all(np.abs(sh) <= 149)
    # the generator's truth is recovered at q_true and overall
    assert tuple(sh[p.true_index]) == p.t_zyx
    assert int(np.argmax(sc)) == p.true_index
    score, ri, chi = f.align(dev(p.B), dev(p.MB), p.quats)
    assert ri == p.true_index and chi == p.t_zyx
    # sampled rotations against the oracle's full map (FFT form at 320^3)
    for r, omap in oracle150.items():
        check_best_against_map(omap, sc[r], sh[r], tau=tau)
    f.release()


@pytest.mark.parametrize("precision,tau", [("fp32", 1e-4), ("bf16", 1e-2), ("fp16", 1e-2)])
def test_150_cubed_whole_maps_at_bound_limited_lengths(cs, pair150, oracle150, precision, tau):
    """Eq. 5 for every shift of the 150^3 pair, element by element against the
    oracle's full-length map, at the lengths the bench runs most rotations at
    (bound-limited, e.g. 200 per axis with n = 150 > P/2: the unpruned first
    stage and the shared-memory NGF slots of the x pass, the two-field z
    pass).  The valid sets must be identical and the error within tau of the
    largest score."""
    p = pair150
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), precision=precision)
    B, MB = dev(p.B), dev(p.MB)
    for r, omap in oracle150.items():
        gmap = f.score_map(B, MB, p.quats[r]).cpu().numpy()
        assert all(v < 320 for v in f.pad) and max(f.pad) < 2 * 150 - 1, f.pad
        assert 2 * 150 > min(f.pad)             # n > P/2 on some axis: unpruned first stage
        check_maps(omap, gmap, tau)
    f.release()


@pytest.fixture(scope="module")
def pair256():
    return synth.config_pair(4)


def test_256_cubed_5000_rotations_fp32_and_fp16(cs, pair256):
    """The 256^3 pair with 5000 rotations in the bench's launch configuration
    (memory-sized batch), in FP32 and in the FP16 form.  All rotations are
    checked by properties; the true and one sampled rotation by the oracle's
    direct sum (Eq. 5) at the GPU's shift and its face neighbours."""
    p = pair256
    R = len(p.quats)
    assert R == 5000
    B, MB = dev(p.B), dev(p.MB)
    res = {}
    for precision in ("fp32", "fp16"):
        f = cs.prepare_fixed(dev(p.A), dev(p.MA), precision=precision)
        sc, sh = [t.cpu().numpy() for t in f.score_rotations(B, MB, p.quats)]
        assert f.max_pad == (512, 512, 512)
        f.release()
        assert sc.shape == (R,) and sh.shape == (R, 3)
        fin = np.isfinite(sc)
        assert fin.all()
        assert sc.min() >= -1e-6 and sc.max() <= 1 + 1e-6
        assert np.all(np.abs(sh) <= 255)
        assert int(np.argmax(sc)) == p.true_index
        assert tuple(sh[p.true_index]) == p.t_zyx
        res[precision] = (sc, sh)
    # FP16 against FP32: the same global argmax, scores within the form's tolerance
    assert float(np.max(np.abs(res["fp16"][0] - res["fp32"][0]))) <= 1e-2
    rng = np.random.default_rng(256)
    sample = [p.true_index] + [int(i) for i in rng.choice(R, 1, replace=False)]
    for r in sample:
        Bh, Mh = O.resample(p.B, p.MB, p.quats[r])
        chis = set()
        for precision in res:
            chis.update(face_neighbours(res[precision][1][r]))
        chis = [c for c in chis if all(abs(v) <= 255 for v in c)]
        omap, _ = O.csngf_direct(p.A, p.MA, Bh, Mh, 1e-5, 0.5, chis=chis)
        check_best_at_sampled_shifts(omap, res["fp32"][0][r], res["fp32"][1][r], tau=1e-4)
        check_best_at_sampled_shifts(omap, res["fp16"][0][r], res["fp16"][1][r], tau=1e-2)
