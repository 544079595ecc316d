"""Continuous-batching server: jobs of different N, d, kernel and k give the
same factor alone and in a mix where they overlap on the GPU; admission
respects the memory budget; bad requests are refused."""
import os
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_03969_gb300 as rp
    rp.lib()
    return rp


def _jobs(count=6, seed=11):
    jobs = workloads.serving_stream(seed, jobs=count, rate_per_s=1000.0, n_lo=1000, n_hi=20000,
                                    k_lo=50, k_hi=300)
    return [(j.problem, 900 + i) for i, j in enumerate(jobs)]


def _run_all(rp, jobs, slots, budget=8 << 30):
    out = []
    with rp.Server(budget, slots) as srv:
        tickets = [srv.submit(p.X, p.kernel, p.sigma, p.k, seed=s) for p, s in jobs]
        for (p, _), t in zip(jobs, tickets):
            r = srv.poll(t, wait_ms=-1)
            assert r["state"] == "finished", r
            F, P = srv.copy_factor(t, p.N, r["rank"])
            out.append((r, F, P))
            srv.release(t)
    return out


def test_results_are_the_same_alone_and_in_the_mix(rp):
    jobs = _jobs()
    alone = _run_all(rp, jobs, slots=1)       # one job on the GPU at a time
    mixed = _run_all(rp, jobs, slots=len(jobs))  # all admitted at once, overlapping
    for (ra, Fa, Pa), (rm, Fm, Pm), (p, _) in zip(alone, mixed, jobs):
        assert ra["rank"] == rm["rank"] == p.k
        assert np.array_equal(Pa, Pm)
        assert np.array_equal(Fa, Fm)  # bit-identical: no cross-job interference
        assert ra["trace_error"] == rm["trace_error"]
    # in the mix, later jobs did not wait for earlier ones to finish
    assert max(r["queue_ms"] for r, _, _ in mixed) < sum(r["run_ms"] for r, _, _ in alone)


def test_admission_respects_the_memory_budget(rp):
    jobs = _jobs(5, seed=12)
    need = [rp.context_bytes(p.N, p.d, p.k, min(120, p.N), "mixed") for p, _ in jobs]
    budget = sorted(need)[-1] + sorted(need)[-2]  # at most two of the largest at once
    with rp.Server(budget, 8) as srv:
        tickets = [srv.submit(p.X, p.kernel, p.sigma, p.k, seed=s) for p, s in jobs]
        peak = 0
        deadline = time.time() + 120
        while time.time() < deadline:
            st = [srv.poll(t) for t in tickets]
            held = sum(r["device_bytes"] for r in st if r["state"] in ("running", "finished"))
            peak = max(peak, held)
            assert held <= budget
            done = [t for t, r in zip(tickets, st) if r["state"] == "finished"]
            for t in done:
                srv.release(t)
                tickets.remove(t)
            if not tickets:
                break
            time.sleep(0.001)
        assert not tickets, "jobs did not finish"
        assert peak > 0


def test_bad_requests(rp):
    p, s = _jobs(1)[0]
    with rp.Server(1 << 30, 2) as srv:
        with pytest.raises(rp.RpcholError):
            srv.submit(p.X, p.kernel, -1.0, p.k)  # sigma <= 0
        with pytest.raises(rp.RpcholError):
            srv.submit(p.X, p.kernel, p.sigma, p.N + 1)  # k > N
        with rp.Server(1024, 1) as tiny:
            with pytest.raises(rp.RpcholError):
                tiny.submit(p.X, p.kernel, p.sigma, p.k)  # can never fit the budget
        t = srv.submit(p.X, p.kernel, p.sigma, p.k, seed=s)
        r = srv.poll(t, wait_ms=-1)
        assert r["state"] == "finished" and r["latency_ms"] >= r["run_ms"] > 0
        srv.release(t)
        with pytest.raises(rp.RpcholError):
            srv.poll(t)  # released
