"""Serving: Poisson arrivals of 3D jobs of mixed sizes, admitted by a
device-memory budget into one resident engine that batches them round by
round (continuous batching).  Each job's result in the mix must equal its
result alone: the oracle's DT of its points (integer output: bit-exact)."""
import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


def _jobs(count, seed, lo, hi, rate):
    from paper_1902_07554_gb300.serve import Job, poisson_arrivals
    sizes, kinds, seeds = pointsets.serve_jobs(count, seed=seed, lo=lo, hi=hi)
    arr = poisson_arrivals(count, rate, seed)
    return [Job(float(arr[i]), i, pointsets.job_points(sizes[i], kinds[i], seeds[i])) for i in range(count)]


def test_results_in_the_mix_equal_results_alone():
    from paper_1902_07554_gb300.serve import Server
    jobs = _jobs(24, 11, 1000, 300_000, rate=40.0)
    srv = Server(budget_bytes=6e9)
    summary = srv.run(jobs)
    assert summary["jobs"] == 24 and summary["failed"] == 0
    assert summary["p99_ms"] >= summary["p50_ms"] > 0 and summary["quanta"] > 1
    res = {r.jid: r for r in srv.results()}
    for j in jobs:
        assert np.array_equal(res[j.jid].simplices.astype(np.int64), oracle.delaunay(j.points)), j.jid


def test_admission_respects_the_budget():
    """The stream is sized from the budget with the measured per-point cost,
    and the points in flight never exceed it."""
    from paper_1902_07554_gb300.serve import Server, calibrate
    fixed, per_point = calibrate(0, 3)
    assert per_point > 0 and fixed > 0
    budget = fixed + per_point * 80_000
    jobs = _jobs(16, 3, 1000, 40_000, rate=1000.0)        # everything arrives at once
    srv = Server(budget_bytes=budget, model=(fixed, per_point), keep_results=False)
    assert srv.capacity == 80_000
    s = srv.run(jobs)
    assert s["failed"] == 0 and s["peak_running_points"] <= srv.capacity
    assert s["device_gb"] * 1e9 <= budget * 1.01


def test_large_job_in_the_mix_matches_oracle():
    """A 1.5M-point clustered 3D job served among smaller ones that arrive
    while it runs equals the oracle's DT of that job, element by element."""
    from paper_1902_07554_gb300.serve import Job, Server
    big = pointsets.job_points(1_500_000, "clustered", 12345)
    jobs = [Job(0.0, 0, big)]
    sizes, kinds, seeds = pointsets.serve_jobs(10, seed=21, lo=1000, hi=100_000)
    for i in range(10):
        jobs.append(Job(0.01 * (i + 1), i + 1, pointsets.job_points(sizes[i], kinds[i], seeds[i])))
    srv = Server(budget_bytes=12e9)
    summary = srv.run(jobs)
    assert summary["jobs"] == 11 and summary["failed"] == 0
    res = {r.jid: r for r in srv.results()}
    assert np.array_equal(res[0].simplices.astype(np.int64), oracle.delaunay(big))
    for j in jobs[1:]:
        assert np.array_equal(res[j.jid].simplices.astype(np.int64), oracle.delaunay(j.points)), j.jid
