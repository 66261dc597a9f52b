"""The allocation-free entry point (cs_ngf_score_rotations_noalloc) against the
handle-based entry point (cs_ngf_prepare_fixed + cs_ngf_score_rotations).

The allocation-free entry point is for callers that cannot call cudaMalloc:
code inside another framework's memory pool or allocator hooks, real-time
loops, processes under a fixed device-memory budget.  Its scratch is a static
device array shared by every call, so these tests make two calls in a row with
different sizes: the second call must not see the first call's leftovers.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth
from tests.parity_util import TAU_FP32, check_best_against_map

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


def _compare_with_handle(cs, p, eps=1e-5, gamma=0.5):
    A, MA, B, MB = dev(p.A), dev(p.MA), dev(p.B), dev(p.MB)
    na_s, na_c = cs.score_rotations_noalloc(A, MA, B, MB, p.quats, eps=eps, gamma=gamma)
    torch.cuda.synchronize()
    f = cs.prepare_fixed(A, MA, eps=eps, gamma=gamma)
    h_s, h_c = f.score_rotations(B, MB, p.quats)
    na_s, na_c = na_s.cpu().numpy(), na_c.cpu().numpy()
    h_s, h_c = h_s.cpu().numpy(), h_c.cpu().numpy()
    scale = float(np.max(np.abs(h_s[np.isfinite(h_s)])))
    assert np.array_equal(np.isfinite(na_s), np.isfinite(h_s))
    fin = np.isfinite(h_s)
    assert np.max(np.abs(na_s[fin] - h_s[fin])) <= TAU_FP32 * scale
    for r in range(len(p.quats)):
        if tuple(na_c[r]) != tuple(h_c[r]):
            # only a near-tie may move the argmax: check the handle path's own
            # map scores the other shift within the tolerance
            m = f.score_map(B, MB, p.quats[r]).cpu().numpy()
            idx = tuple(int(c) + n - 1 for c, n in zip(na_c[r], p.A.shape))
            assert abs(float(m[idx]) - float(h_s[r])) <= TAU_FP32 * scale
    f.release()
    return na_s, na_c


def test_noalloc_matches_handle_path_on_two_calls_in_a_row(cs):
    p1 = synth.config_pair(0)                                  # 32^3, 8 rotations
    p2 = synth.small_pair(77, (20, 17, 23), n_rot=5)           # different size next
    s1, c1 = _compare_with_handle(cs, p1)
    s2, c2 = _compare_with_handle(cs, p2)
    assert c1[p1.true_index].tolist() == list(p1.t_zyx)
    # and the first problem again, after the scratch held the second one
    s3, c3 = _compare_with_handle(cs, p1)
    np.testing.assert_array_equal(s1, s3)
    np.testing.assert_array_equal(c1, c3)


def test_noalloc_rejects_sizes_beyond_its_scratch(cs):
    rng = np.random.default_rng(0)
    dims = (8, 33, 8)
    A = dev(rng.random(dims).astype(np.float32))
    M = dev(np.ones(dims, np.uint8))
    with pytest.raises(cs.CsNgfError) as e:
        cs.score_rotations_noalloc(A, M, A, M, [[1.0, 0, 0, 0]])
    assert e.value.status == cs.EINVAL
    assert "32" in str(e.value)


def _compare_with_oracle(cs, p, eps=1e-5, gamma=0.5):
    """Per rotation, the gap rule against the FP64 oracle's full map."""
    sc, sh = cs.score_rotations_noalloc(dev(p.A), dev(p.MA), dev(p.B), dev(p.MB), p.quats,
                                        eps=eps, gamma=gamma)
    sc, sh = sc.cpu().numpy(), sh.cpu().numpy()
    kinds = []
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, eps=eps, gamma=gamma)
        kinds.append(check_best_against_map(omap, sc[r], sh[r], tau=TAU_FP32))
    return kinds


def test_noalloc_against_the_oracle_32_cubed_and_ragged(cs):
    kinds = _compare_with_oracle(cs, synth.config_pair(0))
    assert kinds.count("exact") >= 6
    kinds = _compare_with_oracle(cs, synth.small_pair(78, (20, 17, 23), n_rot=4))
    assert "exact" in kinds


@pytest.mark.parametrize("dims", [(8, 5, 12), (2, 16, 3), (16, 9, 2)])
def test_noalloc_every_fft_length_against_handle_and_oracle(cs, dims):
    """Mixed small sizes, so that the 16-, 32- and 64-point arms of the
    allocation-free path all run (2n - 1 <= 16, <= 32, <= 64), including the
    smallest size (2) on an axis."""
    p = synth.small_pair(200 + sum(dims), dims, n_rot=4, masks="full", max_shift=1)
    _compare_with_handle(cs, p)
    _compare_with_oracle(cs, p)

