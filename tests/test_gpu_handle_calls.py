"""Calls on one handle: a second host thread is refused with CS_NGF_EBUSY while
a call runs, and calls on different streams are ordered on the handle's
buffers (each waits for the previous call's work), so their results equal
those of the same calls made one after another on one stream."""
import threading
import time

import numpy as np
import pytest

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


def test_second_thread_gets_ebusy_while_a_call_runs(cs):
    # the 150^3 pair and its 1000 rotations: the synchronous host-buffer call
    # runs for a few hundred milliseconds
    p = synth.config_pair(1)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=32)
    B, MB = np.ascontiguousarray(p.B), np.ascontiguousarray(p.MB)
    dB, dMB = dev(p.B), dev(p.MB)
    want_s, want_c = f.score_rotations_host(B, MB, p.quats)
    # a call's launch groups (mask pairs, length classes) depend on its own
    # rotations, so a shorter call is compared with the same shorter call
    want8 = f.score_rotations_host(B, MB, p.quats[:8])
    entered, out = threading.Event(), {}

    def long_call():
        entered.set()
        out["r"] = f.score_rotations_host(B, MB, p.quats)

    t = threading.Thread(target=long_call)
    t.start()
    entered.wait()
    time.sleep(0.05)
    busy_seen, others = 0, []
    while t.is_alive():
        try:
            f.score_map(dB, dMB, p.quats[0])
            others.append("ok")
        except cs.CsNgfError as e:
            if e.status == cs.EBUSY:
                busy_seen += 1
            else:
                others.append(e.status)
        time.sleep(0.01)
    t.join()
    assert busy_seen >= 1
    assert all(o == "ok" for o in others), others
    # the refused calls left the running one alone
    s, c = out["r"]
    np.testing.assert_array_equal(s, want_s)
    np.testing.assert_array_equal(c, want_c)
    # and the handle is free again
    s2, c2 = f.score_rotations_host(B, MB, p.quats[:8])
    np.testing.assert_array_equal(s2, want8[0])
    np.testing.assert_array_equal(c2, want8[1])
    f.release()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_calls_on_two_streams_are_ordered(cs, precision):
    p = synth.small_pair(31, (40, 36, 44), n_rot=24)
    q = synth.small_pair(32, (40, 36, 44), n_rot=24)
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=8, precision=precision)
    B1, M1, B2, M2 = dev(p.B), dev(p.MB), dev(q.B), dev(q.MB)
    # one after another on one stream
    w1 = [t.clone() for t in f.score_rotations(B1, M1, p.quats)]
    w2 = [t.clone() for t in f.score_rotations(B2, M2, q.quats)]
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        # the second call is enqueued on another stream while the first call's
        # kernels are still in flight
        g1 = f.score_rotations(B1, M1, p.quats, stream=s1)
        g2 = f.score_rotations(B2, M2, q.quats, stream=s2)
        s1.synchronize()
        s2.synchronize()
        for got, want in ((g1, w1), (g2, w2)):
            assert torch.equal(got[0], want[0])
            assert torch.equal(got[1], want[1])
    f.release()
