"""Serving loop: continuous batching of submitted requests.

Requests submitted while others run are admitted as memory allows, share the
same launches, and each result is identical to the same request run alone
(per-job random streams and fixed-order reductions; tolerance 0)."""
import numpy as np
import pytest

from paper_2604_03271_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for i in range(6):
        if i % 2 == 0:
            s = W.gaussian_small(i + 1)
            o = W.Options(particles=512 * (1 + i % 3), sweeps=3, seed=100 + i)
        else:
            s = W.xps_like(i, n=400, k_true=2, k_max=3)
            o = W.Options(particles=1024, sweeps=2, seed=200 + i)
        out.append((s, o))
    return out


def test_served_results_equal_alone_results():
    from paper_2604_03271_b300 import api
    reqs = _requests()
    with api.Context(0) as ctx:
        alone = [ctx.run(s, o, keep_samples=False) for s, o in reqs]
        jobs = []
        for s, o in reqs:
            jobs.append(ctx.submit(s, o))
        for j in jobs:
            ctx.wait(j, 120.0)
        served = []
        for j, (s, _) in zip(jobs, reqs):
            served.append(ctx.result(j, s))
            ctx.release(j)
    for a, b in zip(alone, served):
        assert b["status"] == 0
        np.testing.assert_array_equal(a["log_z"], b["log_z"])
        np.testing.assert_array_equal(a["n_stages"], b["n_stages"])
        for x, y in zip(a["post_mean"], b["post_mean"]):
            np.testing.assert_array_equal(x, y)
        assert b["latency_ms"] > 0


def test_served_requests_share_launches():
    # continuous batching: requests in flight together advance in the same
    # kernel launches (the profile counts the most requests in one launch)
    from paper_2604_03271_b300 import api
    reqs = _requests()
    with api.Context(0) as ctx:
        ctx.profile_reset()
        jobs = ctx.submit_batch(reqs)
        for j in jobs:
            ctx.wait(j, 120.0)
        for j, (s, _) in zip(jobs, reqs):
            assert ctx.result(j, s)["status"] == 0
            ctx.release(j)
        assert ctx.profile()["max_batch_requests"] >= 2


def test_admission_by_memory_budget():
    # Three or more requests queued together, with a budget that holds exactly
    # one of them: admission must add up what it admits in one pass, so they
    # run one after another and all succeed (none fails for lack of memory).
    from paper_2604_03271_b300 import api
    s, _ = _requests()[1]
    reqs = [(s, W.Options(particles=1024, sweeps=2, seed=300 + i)) for i in range(4)]
    with api.Context(0) as probe:
        need = probe.request_bytes(*reqs[0])
    budget = need + need // 2
    assert need > budget // 2  # two never fit together
    with api.Context(0, mem_budget_bytes=budget) as ctx:
        ctx.profile_reset()
        jobs = ctx.submit_batch(reqs)
        for j in jobs:
            ctx.wait(j, 120.0)
        for j, (sp, _) in zip(jobs, reqs):
            r = ctx.result(j, sp)
            assert r["status"] == 0, r["status"]
            ctx.release(j)
        assert ctx.profile()["max_batch_requests"] == 1
    # the same requests alone: identical results (admission order changes nothing)
    with api.Context(0) as ctx:
        ref = ctx.run(*reqs[2], keep_samples=False)
    with api.Context(0, mem_budget_bytes=budget) as ctx:
        jobs = ctx.submit_batch(reqs)
        for j in jobs:
            ctx.wait(j, 120.0)
        got = ctx.result(jobs[2], reqs[2][0])
        for j in jobs:
            ctx.release(j)
    np.testing.assert_array_equal(ref["log_z"], got["log_z"])


def test_admission_waits_for_budget_held_by_served_requests():
    # submitted one by one while earlier ones run: a request that does not fit
    # yet waits for memory instead of failing
    from paper_2604_03271_b300 import api
    reqs = _requests()[:4]
    with api.Context(0) as probe:
        need = max(probe.request_bytes(s, o) for s, o in reqs)
    with api.Context(0, mem_budget_bytes=need + need // 2) as ctx:
        jobs = [ctx.submit(s, o) for s, o in reqs]
        for j in jobs:
            ctx.wait(j, 120.0)
        for j, (s, _) in zip(jobs, reqs):
            r = ctx.result(j, s)
            assert r["status"] == 0
            ctx.release(j)


def test_oversized_request_fails_cleanly():
    from paper_2604_03271_b300 import api
    s, o = W.gaussian_small(1), W.Options(particles=1 << 20, sweeps=2, seed=1)
    with api.Context(0, mem_budget_bytes=8 << 20) as ctx:
        j = ctx.submit(s, o)
        ctx.wait(j, 30.0)
        r = ctx.result(j, s)
        assert r["status"] == api.SMC_ENOMEM and r["log_z"] is None
        ctx.release(j)


def test_request_arriving_mid_run_joins_the_running_launches():
    # continuous batching under arrivals: a small request submitted while a
    # large one is on the GPU is admitted at the next stage boundary, shares
    # its launches, and finishes first; submitting does not wait for the
    # serving thread's launches
    import time

    from paper_2604_03271_b300 import api
    big = (W.xrd_like(2, n=2048, k_true=6, k_max=8), W.Options(particles=16384, sweeps=20, seed=5))
    small = (W.gaussian_small(3), W.Options(particles=1024, sweeps=4, seed=6))
    with api.Context(0) as ctx:
        ref_small = ctx.run(*small, keep_samples=False)
        ctx.profile_reset()
        ja = ctx.submit(*big)
        time.sleep(0.3)
        assert not ctx.poll(ja)  # the large request is still running
        t0 = time.perf_counter()
        jb = ctx.submit(*small)
        submit_ms = 1000.0 * (time.perf_counter() - t0)
        ctx.wait(jb, 120.0)
        b_done_first = not ctx.poll(ja)
        ctx.wait(ja, 600.0)
        rb = ctx.result(jb, small[0])
        ra = ctx.result(ja, big[0])
        for j in (ja, jb):
            ctx.release(j)
        assert ra["status"] == 0 and rb["status"] == 0
        assert submit_ms < 100.0, submit_ms
        assert b_done_first
        assert ctx.profile()["max_batch_requests"] >= 2
    np.testing.assert_array_equal(ref_small["log_z"], rb["log_z"])
