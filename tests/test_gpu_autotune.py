"""Autotuned radix splits (cs_ngf_config.autotune): the first launch group at
new FFT lengths times both splits of each pass that has two, keeps the faster
for the process, and the results match the oracle and the built-in splits."""
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


# lengths with a second split (include/cs_ngf.h, fft_core.cuh SplitV)
ALT = {64: (4, 16), 80: (4, 20), 128: (4, 32), 160: (10, 16), 192: (8, 24), 200: (8, 25),
       216: (8, 27), 256: (8, 32), 320: (10, 32), 400: (20, 20)}


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_autotuned_splits_match_oracle_and_default(cs, precision):
    cs.tuning_reset()
    p = synth.small_pair(41, (36, 30, 34), masks="threshold", n_rot=10)
    kw = dict(batch=4, pad_mode="full", precision=precision)      # lengths 80, 64, 80
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), autotune=True, **kw)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    table = cs.tuning()
    timed = {(e["stage"], e["length"]) for e in table}
    assert timed == {("fwd_x", 80), ("fwd_y", 64), ("zmac", 80), ("inv_y", 64), ("inv_x", 80)}
    for e in table:
        assert e["splits"][1] == ALT[e["length"]] and e["splits"][0][0] * e["splits"][0][1] == e["length"]
        assert e["ms"][0] > 0 and e["ms"][1] > 0 and e["variant"] == int(e["ms"][1] < e["ms"][0])
    tau = TAU_FP32 if precision == "fp32" else 1e-2
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_best_against_map(omap, sc[r], sh[r], tau=tau)
    d = cs.prepare_fixed(dev(p.A), dev(p.MA), **kw)                # built-in splits
    sd, _ = [t.cpu().numpy() for t in d.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert np.max(np.abs(sd - sc)) <= tau * np.max(np.abs(sd))
    # the choices are kept: another autotuned handle does not time again and
    # gives the same results bit for bit
    g = cs.prepare_fixed(dev(p.A), dev(p.MA), autotune=True, **kw)
    sg, cg = [t.cpu().numpy() for t in g.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert cs.tuning() == table
    np.testing.assert_array_equal(sg, sc)
    np.testing.assert_array_equal(cg, sh)
    # and so does the first handle's next call, which replays its graphs
    s2, c2 = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    np.testing.assert_array_equal(s2, sc)
    np.testing.assert_array_equal(c2, sh)


def test_autotune_with_bound_limited_lengths(cs):
    """Several length classes in one call: each new set of lengths is timed on
    its first launch group."""
    cs.tuning_reset()
    p = synth.small_pair(21, (30, 30, 30), masks="threshold", n_rot=48)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4, autotune=True)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    lengths = {ln for cp, _ in f.length_classes() for ln in cp}
    timed = {e["length"] for e in cs.tuning()}
    assert {ln for ln in lengths if ln in ALT} <= timed
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_best_against_map(omap, sc[r], sh[r])


@pytest.mark.parametrize("P", sorted(ALT))
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_every_alternative_split_matches_oracle(cs, P, axis):
    """Each length's second split on one axis at a time (z: the z pass; y: the
    y forward and inverse passes; x: the x forward and inverse passes), full
    padding so that the length is the requested one, against the oracle."""
    dims = (7, 8, 6)
    pad = [16, 16, 16]
    pad[axis] = P
    p = synth.small_pair(900 + P + axis, dims, masks="threshold", n_rot=2)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), pad=tuple(pad), pad_mode="full", autotune="alternative")
    for q in (p.q_true, p.quats[-1]):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=tuple(pad))
        check_maps(omap, gmap)
    f.release()


def test_alternative_splits_with_full_length_inputs(cs):
    """Bound-limited lengths shorter than twice the side, so that the forward
    passes read full-length inputs, with every alternative split."""
    p = synth.small_pair(21, (30, 30, 30), masks="threshold", n_rot=24)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4, autotune="alternative")
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert any(ln in ALT for cp, _ in f.length_classes() for ln in cp)
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_best_against_map(omap, sc[r], sh[r])
