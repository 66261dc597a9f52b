"""Serving loop: jobs of mixed sizes arriving while others run give the same
results as scoring each job alone; admission by memory; cancel; a host-side
injected admission failure leaves the other jobs correct."""
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


def alone(cs, p, quats, batch):
    f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=batch)
    sc, sh = f.score_rotations(dev(p.B), dev(p.MB), quats)
    out = sc.cpu().numpy(), sh.cpu().numpy()
    f.release()
    return out


def make_jobs(n, seed):
    rng = np.random.default_rng(seed)
    shapes = [(20, 24, 22), (24, 24, 24), (16, 28, 20), (30, 18, 26)]
    pairs = {s: synth.small_pair(100 + i, s, n_rot=2) for i, s in enumerate(shapes)}
    jobs = []
    for k in range(n):
        s = shapes[int(rng.integers(len(shapes)))]
        R = int(rng.integers(5, 40))
        q = synth.random_quaternions(rng, R)
        jobs.append((pairs[s], q))
    return jobs


def test_mixed_jobs_equal_alone(cs):
    batch = 8
    jobs = make_jobs(14, 1)
    srv = cs.Server(max_active_jobs=3, max_inflight=2, batch=batch)
    rng = np.random.default_rng(2)
    ids = []
    for p, q in jobs:                      # Poisson-like arrivals while earlier jobs run
        ids.append(srv.submit(p.A, p.MA, p.B, p.MB, q))
        time.sleep(float(rng.exponential(0.002)))
    results = [srv.wait(j, timeout_s=120) for j in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["pending"] == 0 and st["active"] == 0
    for (p, q), res in zip(jobs, results):
        assert res["status"] == cs.OK
        sc, sh = alone(cs, p, q, batch)
        np.testing.assert_array_equal(res["scores"], sc)
        np.testing.assert_array_equal(res["shifts"], sh)
        best = int(np.argmax(sc))
        assert res["rot_index"] == best and res["score"] == sc[best]
        assert res["latency_ms"] >= res["queue_ms"] >= 0


def test_tight_memory_budget_still_serves_every_job(cs):
    """A budget that holds only about one job's resources: the server must
    evict idle pooled resources of other shapes and admit jobs one by one."""
    jobs = make_jobs(5, 3)
    need = 0
    for p, q in jobs:
        f = cs.prepare_fixed(dev(p.A), dev(p.MA), batch=8)
        need = max(need, f.fixed_bytes + f.workspace_bytes + 10 * p.A.size + 16 * len(q) + (1 << 16))
        f.release()
    srv = cs.Server(memory_budget_bytes=int(need * 1.2), max_active_jobs=4, batch=8)
    ids = [srv.submit(p.A, p.MA, p.B, p.MB, q) for p, q in jobs]
    res = [srv.wait(j, timeout_s=120) for j in ids]
    st = srv.stats()
    srv.close()
    assert st["bytes_in_use"] <= st["memory_budget_bytes"]
    for (p, q), r in zip(jobs, res):
        assert r["status"] == cs.OK
        sc, _ = alone(cs, p, q, 8)
        np.testing.assert_array_equal(r["scores"], sc)


def test_job_larger_than_budget_is_refused(cs):
    p, q = make_jobs(1, 4)[0]
    srv = cs.Server(memory_budget_bytes=1 << 20, batch=8)
    with pytest.raises(cs.CsNgfError) as e:
        srv.submit(p.A, p.MA, p.B, p.MB, q)
    assert e.value.status == cs.ENOMEM
    srv.close()


def test_cancel_and_injected_failure_leave_others_correct(cs):
    jobs = make_jobs(6, 5)
    srv = cs.Server(max_active_jobs=1, batch=8, inject_admission_failure=3)
    ids = [srv.submit(p.A, p.MA, p.B, p.MB, q) for p, q in jobs]
    srv.cancel(ids[5])                      # still pending behind the others
    res = [srv.wait(j, timeout_s=120) for j in ids]
    srv.close()
    assert res[2]["status"] == cs.ENOMEM    # job id 3: injected admission failure
    assert res[5]["status"] == cs.ECANCELED and res[5]["scored"] == 0
    for k in (0, 1, 3, 4):
        p, q = jobs[k]
        sc, sh = alone(cs, p, q, 8)
        assert res[k]["status"] == cs.OK
        np.testing.assert_array_equal(res[k]["scores"], sc)
        np.testing.assert_array_equal(res[k]["shifts"], sh)


@pytest.mark.parametrize("policy", ["arrival", "shortest"])
def test_admission_policy_order(cs, policy):
    """One active slot: a long job runs while a long and then a short job wait.
    Arrival order admits the long one first; shortest expected work first
    admits the short one first.  Results equal scoring each job alone."""
    batch = 8
    rng = np.random.default_rng(7)
    big = synth.small_pair(301, (64, 64, 64), n_rot=2)
    small = synth.small_pair(302, (16, 16, 16), n_rot=2)
    q_run = synth.random_quaternions(rng, 400)
    q_big = synth.random_quaternions(rng, 200)
    q_small = synth.random_quaternions(rng, 8)
    srv = cs.Server(max_active_jobs=1, max_inflight=2, batch=batch, policy=policy)
    j_run = srv.submit(big.A, big.MA, big.B, big.MB, q_run)
    j_big = srv.submit(big.A, big.MA, big.B, big.MB, q_big)
    j_small = srv.submit(small.A, small.MA, small.B, small.MB, q_small)
    r_run, r_big, r_small = (srv.wait(j, timeout_s=300) for j in (j_run, j_big, j_small))
    srv.close()
    assert r_run["status"] == r_big["status"] == r_small["status"] == cs.OK
    if policy == "arrival":
        assert r_big["queue_ms"] < r_small["queue_ms"]
    else:
        assert r_small["queue_ms"] < r_big["queue_ms"]
    for p, q, r in ((big, q_big, r_big), (small, q_small, r_small)):
        sc, sh = alone(cs, p, q, batch)
        np.testing.assert_array_equal(r["scores"], sc)
        np.testing.assert_array_equal(r["shifts"], sh)


def test_unknown_policy_is_refused(cs):
    with pytest.raises(ValueError):
        cs.Server(policy="fastest")
