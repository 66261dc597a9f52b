"""Host logic of bound-limited padding (cs_ngf_plan_lengths, no GPU): the
lengths each rotation needs, their classes and the merge rule, against a
plain mirror of the rule and against the alias-free condition."""
import numpy as np
import pytest

# supported FFT lengths (include/cs_ngf.h)
PADS = (16, 32, 40, 64, 80, 100, 128, 160, 192, 200, 216, 256, 320, 360, 400, 512)


@pytest.fixture(scope="module")
def binding():
    try:
        from paper_2110_10156_gb300 import cs_ngf
    except (ImportError, OSError) as e:
        pytest.skip(f"library not built: {e}")
    return cs_ngf


def auto_pad(n):
    return min(v for v in PADS if v >= 2 * n - 1)


def needs(dims, max_pad, b):
    """Per axis the shortest supported P >= n + max(-chi_lo, chi_hi) (slots
    v = chi + n - 1), at most max_pad; None if some axis admits no shift."""
    if b[0] > b[1] or b[2] > b[3] or b[4] > b[5]:
        return None
    out = []
    for a, n in enumerate(dims):
        lo, hi = b[2 * a] - (n - 1), b[2 * a + 1] - (n - 1)
        out.append(min(min(v for v in PADS if v >= n + max(-lo, hi)), max_pad[a]))
    return tuple(out)


def mirror(dims, max_pad, bounds, cur=(0, 0, 0), class_cost=4.0, max_classes=8):
    per = [needs(dims, max_pad, b) for b in bounds]
    cls, none = {}, []
    for r, t in enumerate(per):
        if t is None:
            none.append(r)
        else:
            cls.setdefault(t, []).append(r)
    cls = [[list(k), v] for k, v in cls.items()]
    vol = lambda t: t[0] * t[1] * t[2]
    while len(cls) > 1:
        best = None
        for c in range(len(cls)):
            for d in range(c + 1, len(cls)):
                m = [max(x, y) for x, y in zip(cls[c][0], cls[d][0])]
                cost = (vol(m) - vol(cls[c][0])) * len(cls[c][1]) + (vol(m) - vol(cls[d][0])) * len(cls[d][1])
                if best is None or cost < best[0]:
                    best = (cost, c, d, m)
        cost, c, d, m = best
        if cost >= class_cost * min(vol(cls[c][0]), vol(cls[d][0])) and len(cls) <= max_classes:
            break
        cls[c][0] = m
        cls[c][1] = sorted(cls[c][1] + cls[d][1])
        del cls[d]
    if not cls:
        cls = [[[min(v for v in PADS if v >= n) for n in dims], []]]
    cls[0][1] = sorted(cls[0][1] + none)
    cls = sorted(cls, key=lambda c: (tuple(c[0]) != tuple(cur), -len(c[1])))     # stable
    return [(tuple(c[0]), len(c[1])) for c in cls], [r for c in cls for r in c[1]], per


def random_bounds(rng, dims, R, spread):
    b = np.zeros((R, 6), np.int32)
    for a, n in enumerate(dims):
        c = n - 1 + rng.integers(-spread // 3, spread // 3 + 1, size=R)
        w = rng.integers(0, spread, size=(R, 2))
        b[:, 2 * a] = np.clip(c - w[:, 0], 0, 2 * n - 2)
        b[:, 2 * a + 1] = np.clip(c + w[:, 1], 0, 2 * n - 2)
    return b


@pytest.mark.parametrize("seed", range(6))
def test_classes_match_the_rule_and_cover_every_rotation(binding, seed):
    rng = np.random.default_rng(seed)
    dims = tuple(int(v) for v in rng.integers(20, 160, size=3))
    max_pad = tuple(auto_pad(n) for n in dims)
    R = int(rng.integers(20, 400))
    b = random_bounds(rng, dims, R, spread=int(rng.integers(4, min(dims))))
    b[rng.integers(0, R, size=3), 2] = 2 * dims[1]          # a few rotations admit no shift
    b[:, 3] = np.where(b[:, 2] > 2 * dims[1] - 2, 0, b[:, 3])
    cur = max_pad if seed % 2 else (0, 0, 0)
    cls, order = binding.plan_lengths(dims, max_pad, b, cur_pad=cur)
    want, want_order, per = mirror(dims, max_pad, b.tolist(), cur=cur)
    assert cls == want
    assert order.tolist() == want_order
    assert sorted(order.tolist()) == list(range(R)) and sum(n for _, n in cls) == R
    assert 1 <= len(cls) <= 8
    # every rotation's class covers its own admitted shifts (alias-free)
    k = 0
    for pad, n in cls:
        for r in order[k:k + n]:
            if per[r] is not None:
                assert all(p >= q for p, q in zip(pad, per[r]))
                for a, nn in enumerate(dims):
                    lo, hi = b[r, 2 * a] - (nn - 1), b[r, 2 * a + 1] - (nn - 1)
                    assert pad[a] >= nn + max(-lo, hi) and pad[a] <= max_pad[a]
        k += n


def test_the_150_cubed_ranges_give_192_to_216(binding):
    """A rotation admitting shifts within +-40 on a 150^3 volume needs 190 <= 192
    per axis; one reaching +51 on y needs 201, hence 216 on that axis, and
    one reaching +45 on x needs 195, hence 200 (the 20 rotations left at 192^3
    then join that class: cheaper than a class of their own)."""
    dims, max_pad = (150, 150, 150), (320, 320, 320)
    b = np.tile(np.array([149 - 40, 149 + 40] * 3, np.int32), (64, 1))
    b[:20, 3] = 149 + 51
    cls, order = binding.plan_lengths(dims, max_pad, b)
    assert cls == [((192, 192, 192), 44), ((192, 216, 192), 20)]
    assert sorted(order[44:].tolist()) == list(range(20))
    b[40:, 5] = 149 + 45
    cls, order = binding.plan_lengths(dims, max_pad, b)
    want, want_order, _ = mirror(dims, max_pad, b.tolist())
    assert cls == want and order.tolist() == want_order
    assert ((192, 192, 200), 44) in cls


def test_bad_arguments(binding):
    b = np.zeros((1, 6), np.int32)
    with pytest.raises(binding.CsNgfError):
        binding.plan_lengths((10, 10, 10), (16, 32, 32), b)          # 16 < 2n - 1
    with pytest.raises(binding.CsNgfError):
        binding.plan_lengths((10, 10, 10), (96, 32, 32), b)          # unsupported length
