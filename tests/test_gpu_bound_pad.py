"""Bound-limited padding (cs_ngf_pad_mode CS_NGF_PAD_BOUND) against the FP64
oracle, whose maps always use the full linear-correlation length 2n - 1.

Section 3.2 admits a shift only where the overlap reaches gamma times the
smaller mask.  The slab counts of the masks bound the overlap along each
axis, so each call can take the shortest FFT length that keeps every
admitted shift alias-free.  These tests check the lengths the library picks
(predicted here from the oracle's resampled masks), that they are shorter
than 2n - 1, that the forward passes then read inputs longer than half the
transform, and that scores and argmaxes match the oracle and the full-length
mode."""
import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth
from tests.parity_util import check_best_against_map, check_maps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# supported FFT lengths (include/cs_ngf.h)
PADS = (16, 32, 40, 64, 80, 100, 128, 160, 192, 200, 216, 256, 320, 360, 400, 512)
IDENTITY = np.array([1.0, 0.0, 0.0, 0.0])


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


def admitted_range(MA, Mh, gamma):
    """Per axis the shifts chi whose slab bound sum_i min(a_i, b_{i+chi})
    reaches the overlap threshold, as (lo, hi); None if an axis admits none."""
    thr = O.overlap_threshold(int(MA.sum()), int(Mh.sum()), gamma)
    out = []
    for ax in range(3):
        other = tuple(i for i in range(3) if i != ax)
        a = MA.astype(np.int64).sum(axis=other)
        b = Mh.astype(np.int64).sum(axis=other)
        n = len(a)
        ok = [c for c in range(-(n - 1), n)
              if np.minimum(a[max(0, -c):min(n, n - c)], b[max(0, c):min(n, n + c)]).sum() >= thr]
        out.append((min(ok), max(ok)) if ok else None)
    return out


def expected_pads(p, quats, gamma=0.5, MB=None):
    """Per axis the shortest supported length >= n + max(-lo, hi) over the
    shifts admitted for any rotation that admits some shift."""
    MB = p.MB if MB is None else MB
    lo, hi = [None] * 3, [None] * 3
    for q in quats:
        _, Mh = O.resample(p.B, MB, q)
        rg = admitted_range(p.MA, Mh, gamma)
        if any(r is None for r in rg):
            continue
        for a in range(3):
            lo[a] = rg[a][0] if lo[a] is None else min(lo[a], rg[a][0])
            hi[a] = rg[a][1] if hi[a] is None else max(hi[a], rg[a][1])
    pads = []
    for a, n in enumerate(p.A.shape):
        need = n if lo[a] is None else n + max(-lo[a], hi[a])
        pads.append(min(v for v in PADS if v >= need))
    return tuple(pads)


CASES = [(5, (24, 22, 26)), (9, (20, 17, 23)), (11, (33, 40, 30)), (13, (50, 45, 48))]


@pytest.mark.parametrize("seed,dims", CASES)
def test_lengths_shorter_and_scores_match_oracle(cs, seed, dims):
    p = synth.small_pair(seed, dims, masks="threshold", n_rot=6)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    auto = tuple(O.auto_pad(n) for n in dims)
    assert f.max_pad == auto and f.pad_mode == "bound"
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    pads = expected_pads(p, p.quats)
    assert f.pad == pads
    assert all(v <= a for v, a in zip(pads, auto)) and any(v < a for v, a in zip(pads, auto))
    assert any(2 * n > v for n, v in zip(dims, pads))       # inputs longer than P/2
    kinds = []
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)        # full length 2n - 1
        kinds.append(check_best_against_map(omap, sc[r], sh[r]))
    assert kinds.count("exact") >= len(kinds) // 2
    score, ri, chi = f.align(dev(p.B), dev(p.MB), p.quats)
    assert ri == int(np.argmax(sc)) and chi == tuple(int(v) for v in sh[ri])
    f.release()


@pytest.mark.parametrize("seed,dims", CASES[:3])
def test_maps_match_oracle(cs, seed, dims):
    """Every map entry: valid set and scores (the map call bounds its one rotation)."""
    p = synth.small_pair(seed, dims, masks="threshold", n_rot=3)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    for q in (IDENTITY, p.q_true, p.quats[-1]):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        assert f.pad == expected_pads(p, [q])
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_maps(omap, gmap)
    f.release()


@pytest.mark.parametrize("measure,precision,tau", [("squared", "fp32", 1e-4), ("unsquared", "fp32", 1e-4),
                                                   ("squared", "bf16", 1e-2)])
def test_same_results_as_full_length(cs, measure, precision, tau):
    p = synth.small_pair(17, (28, 26, 30), masks="threshold", n_rot=8)
    kw = dict(measure=measure, precision=precision)
    fb = cs.prepare_fixed(dev(p.A), dev(p.MA), pad_mode="bound", **kw)
    ff = cs.prepare_fixed(dev(p.A), dev(p.MA), pad_mode="full", **kw)
    sb, cb = [t.cpu().numpy() for t in fb.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    sf, cf = [t.cpu().numpy() for t in ff.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert fb.pad != ff.pad and ff.pad == ff.max_pad
    np.testing.assert_array_equal(np.isfinite(sb), np.isfinite(sf))
    fin = np.isfinite(sf)
    assert np.max(np.abs(sb[fin] - sf[fin])) <= tau * np.max(np.abs(sf[fin]))
    for r, q in enumerate(p.quats):
        if tuple(cb[r]) != tuple(cf[r]):          # only a near-tie may move the argmax
            omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, measure=measure)
            check_best_against_map(omap, sb[r], cb[r], tau=tau)


def test_lengths_follow_each_call_and_fixed_volume_updates(cs):
    """Calls with other rotation sets or another fixed volume pick their own
    lengths (fixed spectra recomputed); going back gives the first results
    bit for bit."""
    p = synth.small_pair(5, (24, 22, 26), masks="threshold", n_rot=6)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4)
    a = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    pad_a = f.pad
    # another floating mask (half of it cut away) moves the admitted range
    MB2 = p.MB.copy()
    MB2[:, :, : p.MB.shape[2] // 2] = 0
    f.score_rotations(dev(p.B), dev(MB2), p.quats)
    assert f.pad == expected_pads(p, p.quats, MB=MB2)
    b = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert f.pad == pad_a
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    # a new fixed volume: same results as a fresh handle on it
    MA2 = p.MA.copy()
    MA2[: p.MA.shape[0] // 2] = 0
    f.update_fixed(dev(p.A), dev(MA2))
    c = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    g = cs.prepare_fixed(dev(p.A), dev(MA2), batch=4)
    d = [t.cpu().numpy() for t in g.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert f.pad == g.pad
    np.testing.assert_array_equal(c[0], d[0])
    np.testing.assert_array_equal(c[1], d[1])


def test_no_admitted_shift_anywhere(cs):
    p = synth.small_pair(61, (12, 12, 12), n_rot=3)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA))
    zero = np.zeros_like(p.MB)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(zero), p.quats)]
    assert np.all(np.isneginf(sc)) and np.all(sh == 0)
    assert all(v >= n for v, n in zip(f.pad, p.A.shape))


def rotation_lengths(p, q, gamma=0.5):
    _, Mh = O.resample(p.B, p.MB, q)
    rg = admitted_range(p.MA, Mh, gamma)
    if any(r is None for r in rg):
        return None
    return tuple(min(v for v in PADS if v >= n + max(-lo, hi)) for n, (lo, hi) in zip(p.A.shape, rg))


def length_classes(per, class_cost=4.0, max_classes=8):
    """The library's grouping rule: rotations needing the same lengths form a
    class; the cheapest pair merges (lengths raised to cover both) while the
    added transform volume is below class_cost rotations of the smaller one,
    or while there are more than max_classes."""
    cls = {}
    for r, t in enumerate(per):
        if t is not None:
            cls.setdefault(t, []).append(r)
    cls = [[list(k), v] for k, v in cls.items()]
    vol = lambda t: t[0] * t[1] * t[2]
    while len(cls) > 1:
        best = None
        for c in range(len(cls)):
            for d in range(c + 1, len(cls)):
                m = [max(a, b) for a, b in zip(cls[c][0], cls[d][0])]
                cost = (vol(m) - vol(cls[c][0])) * len(cls[c][1]) + (vol(m) - vol(cls[d][0])) * len(cls[d][1])
                if best is None or cost < best[0]:
                    best = (cost, c, d, m)
        cost, c, d, m = best
        if cost >= class_cost * min(vol(cls[c][0]), vol(cls[d][0])) and len(cls) <= max_classes:
            break
        cls[c][0] = m
        cls[c][1] += cls[d][1]
        del cls[d]
    return cls


def test_rotations_grouped_by_their_own_lengths(cs):
    """Each rotation gets the lengths its own admitted shifts need; the call
    scores the classes one after another and returns the results in the
    caller's order.  Every rotation is checked against the oracle, and the
    whole set against the full-length mode."""
    p = synth.small_pair(21, (30, 30, 30), masks="threshold", n_rot=48)
    per = [rotation_lengths(p, q) for q in p.quats]
    cls = length_classes(per)
    assert len(cls) > 2
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    assert f.length_sets == len(cls)
    assert f.pad in {tuple(c[0]) for c in cls}
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q)
        check_best_against_map(omap, sc[r], sh[r])
    ff = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=4, pad_mode="full")
    sf, cf = [t.cpu().numpy() for t in ff.score_rotations(dev(p.B), dev(p.MB), p.quats)]
    fin = np.isfinite(sf)
    np.testing.assert_array_equal(np.isfinite(sc), fin)
    assert np.max(np.abs(sc[fin] - sf[fin])) <= 1e-4 * np.max(np.abs(sf[fin]))
    # a second call with the rotations in reverse order gives the same per-rotation results
    sr, cr = [t.cpu().numpy()[::-1] for t in f.score_rotations(dev(p.B), dev(p.MB), p.quats[::-1])]
    np.testing.assert_allclose(sr, sc, rtol=0, atol=1e-4 * np.max(np.abs(sf[fin])))
    s, ri, chi = f.align(dev(p.B), dev(p.MB), p.quats)
    assert ri == int(np.argmax(sc)) and chi == tuple(int(v) for v in sh[ri])


# Lengths with a factor 3 (192 = 12 x 16, 216 = 12 x 18: the radix-3 register
# DFT) on every axis, with full-length inputs: full masks and gamma = 1/4 admit
# shifts out to 3n/4, so bound-limited padding picks 192 or 216 for n > P/2.
# gamma is exact in FP32 (the ABI's type) and FP64 (the oracle's), so both
# sides take the same threshold ceil(gamma min(sum M_A, sum M_hat)).
RADIX3_CASES = [((104, 10, 12), 0, 192), ((122, 9, 11), 0, 216), ((12, 104, 10), 1, 192),
                ((9, 122, 11), 1, 216), ((10, 12, 104), 2, 192), ((11, 9, 122), 2, 216),
                ((200, 10, 12), 0, 360), ((10, 12, 200), 2, 360)]


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("dims,axis,want", RADIX3_CASES)
def test_radix3_lengths_full_length_inputs(cs, dims, axis, want, precision):
    gamma = 0.25
    p = synth.small_pair(60 + sum(dims), dims, masks="full", n_rot=2)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), gamma=gamma, precision=precision)
    tau = 1e-4 if precision == "fp32" else 1e-2
    for q in (IDENTITY, p.quats[1]):
        gmap = f.score_map(dev(p.B), dev(p.MB), q).cpu().numpy()
        assert f.pad == expected_pads(p, [q], gamma)
        assert f.pad[axis] == want and 2 * dims[axis] > want
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, gamma=gamma)
        check_maps(omap, gmap, tau=tau)
    f.release()
