"""The tensor-core z pass of the reduced-precision forms (k_zx_tc: the
forward z-axis DFT of the channel fields as BF16 / FP16 MMAs with FP32
accumulation in tensor memory, and the Eq. 7-8 sum; k_zinv: the FP32 mask
field and the inverse) against the FP64 oracle, element by element, at every
z length it runs at, through the C ABI.

Each case also scores the same input with the CUDA-core FFT of the same
precision form (tensor_cores=False): the two maps must differ (so the
tensor-core kernel really ran) while both stay within the reduced-precision
tolerance of the oracle with identical valid sets (the overlap count N keeps
its FP32 path)."""
import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from paper_2110_10156_gb300 import synth
from tests.parity_util import check_best_against_map, check_maps

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TAU = 1e-2          # reduced-precision score tolerance, relative to max |s|
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


def rand_quat(seed):
    return synth.random_quaternions(np.random.default_rng(seed), 1)[0]


def run_case(cs, p, pad, pad_mode, precision="bf16", measure="squared", autotune=False, expect_pz=None,
             quats=None):
    A, MA, B, MB = dev(p.A), dev(p.MA), dev(p.B), dev(p.MB)
    kw = dict(pad=pad, precision=precision, pad_mode=pad_mode, measure=measure, autotune=autotune)
    f_tc = cs.prepare_fixed(A, MA, **kw)
    f_cc = cs.prepare_fixed(A, MA, tensor_cores=False, **kw)
    differs, worst = False, 0.0
    quats = quats if quats is not None else (IDENTITY, p.q_true, rand_quat(11))
    pads = []
    for q in quats:
        m_tc = f_tc.score_map(B, MB, q).cpu().numpy()
        m_cc = f_cc.score_map(B, MB, q).cpu().numpy()
        pads.append(tuple(f_tc.pad))
        if expect_pz is not None:
            assert f_tc.pad[0] == expect_pz, f_tc.pad
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=pad, measure=measure)
        worst = max(worst, check_maps(omap, m_tc, tau=TAU))
        check_maps(omap, m_cc, tau=TAU)
        differs |= not np.array_equal(m_tc, m_cc)
    assert differs, "tensor-core and CUDA-core maps are identical: the tensor-core pass did not run"
    f_tc.release()
    f_cc.release()
    run_case.pads = pads
    return worst


# every z length the tensor-core pass takes, half-length inputs (n <= P/2),
# full padding with the lengths given
TC_LENGTH_CASES = [
    ((7, 10, 6), (16, 32, 16)),          # 4 x 4 split: the CUDA-core half has 2 warps
    ((12, 10, 14), (32, 32, 32)),
    ((18, 12, 9), (40, 32, 32)),
    ((30, 10, 12), (64, 32, 32)),
    ((36, 9, 11), (80, 32, 32)),
    ((45, 10, 9), (100, 100, 32)),       # ragged y tail: 100 columns in blocks of 8
    ((60, 8, 10), (128, 16, 32)),
    ((70, 9, 8), (160, 32, 16)),
    ((96, 8, 9), (192, 16, 32)),         # radix-3 CUDA-core half (12 x 16)
    ((90, 8, 9), (200, 16, 32)),         # the 150^3 workload's z length
    ((108, 8, 9), (216, 16, 32)),        # 12 x 18
]


@pytest.mark.parametrize("dims,pad", TC_LENGTH_CASES)
def test_tensor_core_z_pass_every_length(cs, dims, pad):
    p = synth.small_pair(900 + sum(dims), dims, masks="threshold", n_rot=3)
    run_case(cs, p, pad, "full", expect_pz=pad[0])


@pytest.mark.parametrize("dims,pad", [((30, 10, 12), (64, 32, 32)), ((60, 8, 10), (128, 16, 32)),
                                      ((96, 8, 9), (192, 16, 32)), ((90, 8, 9), (200, 16, 32)),
                                      ((108, 8, 9), (216, 16, 32))])
def test_tensor_core_z_pass_alternative_splits(cs, dims, pad):
    """The second radix split of each length (4 x 16, 4 x 32, 8 x 24, 8 x 25,
    8 x 27) changes the CUDA-core half's block (256, 512, 384, 400 and 432
    threads, the 400- and 432-thread blocks with a half warp)."""
    p = synth.small_pair(950 + sum(dims), dims, masks="threshold", n_rot=3)
    run_case(cs, p, pad, "full", autotune="alternative", expect_pz=pad[0])


def ball_pair(seed, dims, radius):
    """A pair whose masks are the same central ball: the overlap bound admits
    only shifts within about the ball's diameter, so bound-limited padding
    picks z lengths below 2n - 1 (n > P/2: the full-length input form)."""
    p = synth.small_pair(seed, dims, masks="full", n_rot=3)
    zz, yy, xx = np.meshgrid(*[np.arange(n) - (n - 1) / 2 for n in dims], indexing="ij")
    ball = ((zz ** 2 + yy ** 2 + xx ** 2) <= radius ** 2).astype(np.uint8)
    p.MA, p.MB = ball.copy(), ball.copy()
    return p


def test_tensor_core_z_pass_full_length_inputs(cs):
    p = ball_pair(971, (36, 12, 12), 4.0)
    run_case(cs, p, None, "bound")
    for pz, _, _ in run_case.pads:          # 40 or 64: below 2n - 1 = 71, with n = 36 > P/2
        assert pz in (40, 64) and 2 * 36 > pz, run_case.pads


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_tensor_core_z_pass_unsquared_measure(cs, precision):
    """Eq. 3 (two channel fields: N = 64 per MMA)."""
    p = synth.small_pair(981, (30, 10, 12), masks="threshold", n_rot=3)
    run_case(cs, p, (64, 32, 32), "full", precision=precision, measure="unsquared", expect_pz=64)


@pytest.mark.parametrize("dims,pad", [((45, 10, 9), (100, 100, 32)), ((90, 8, 9), (200, 16, 32))])
def test_tensor_core_z_pass_fp16(cs, dims, pad):
    """FP16 operands (the per-field power-of-two scale is undone on the
    accumulator): within the tolerance, and closer to the oracle than BF16."""
    p = synth.small_pair(990 + sum(dims), dims, masks="threshold", n_rot=3)
    e16 = run_case(cs, p, pad, "full", precision="fp16", expect_pz=pad[0])
    eb = run_case(cs, p, pad, "full", precision="bf16", expect_pz=pad[0])
    assert 0.0 < e16 < eb


@pytest.mark.parametrize("batch", [4, 6])
def test_tensor_core_batches_with_unpaired_last_rotation(cs, batch):
    """Launch groups of 4 or 6 over 7 rotations: the last group holds one
    rotation whose mask field has no partner, and the two operand stages and
    tensor-memory buffers alternate across an odd count.  Every rotation's
    best shift against the oracle's map (gap rule)."""
    p = synth.small_pair(997, (40, 12, 14), masks="threshold", n_rot=7)
    A, MA, B, MB = dev(p.A), dev(p.MA), dev(p.B), dev(p.MB)
    f = cs.prepare_fixed(A, MA, pad=(80, 32, 32), pad_mode="full", precision="bf16", batch=batch)
    sc, sh = [t.cpu().numpy() for t in f.score_rotations(B, MB, p.quats)]
    for r, q in enumerate(p.quats):
        omap, _ = O.score_map(p.A, p.MA, p.B, p.MB, q, pad=(80, 32, 32))
        check_best_against_map(omap, sc[r], sh[r], tau=TAU)
    score, ri, chi = f.align(B, MB, p.quats)
    assert ri == int(np.argmax(sc)) and score == sc[ri]
    f.release()
