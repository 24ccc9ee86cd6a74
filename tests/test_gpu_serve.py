"""Serving: jobs arriving over time are admitted by a device-memory budget,
small ones batched together, large ones divided, on several concurrent
workers (contexts and streams).  Each job's result in the mix must equal its
result alone: the oracle's DT for small jobs, a standalone library run for
the large ones (integer output: bit-exact)."""
import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


def _jobs(count, seed, lo, hi, rate):
    from paper_1902_07554_gb300.serve import Job, k_for, poisson_arrivals
    sizes, kinds, seeds = pointsets.serve_jobs(count, seed=seed, lo=lo, hi=hi)
    arr = poisson_arrivals(count, rate, seed)
    jobs = []
    for i in range(count):
        P = pointsets.job_points(sizes[i], kinds[i], seeds[i])
        jobs.append(Job(float(arr[i]), i, P, k=k_for(len(P), divide=True), frac=0.005))
    return jobs


def test_results_in_the_mix_equal_results_alone():
    from paper_1902_07554_gb300 import Triangulator
    from paper_1902_07554_gb300.serve import Server
    jobs = _jobs(24, 11, 1000, 300_000, rate=40.0)
    srv = Server(workers=3, budget_bytes=6e9, bytes_per_point=4000.0, small_job=20_000, batch_points=200_000)
    summary = srv.run(jobs)
    assert summary["jobs"] == 24
    assert summary["batched_jobs"] > 0 and summary["p99_ms"] >= summary["p50_ms"] > 0
    res = {r.jid: r for r in srv.results()}
    with Triangulator(0) as alone:
        for j in jobs:
            got = res[j.jid].simplices.astype(np.int64)
            if len(j.points) <= 20_000:
                want = oracle.delaunay(j.points)
            else:
                want = alone.triangulate(j.points, k=j.k, sample_frac=j.frac).astype(np.int64)
            assert np.array_equal(got, want), j.jid


def test_admission_respects_the_budget():
    from paper_1902_07554_gb300.serve import Server
    jobs = _jobs(16, 3, 1000, 40_000, rate=1000.0)        # everything arrives at once
    budget = 4000.0 * 60_000 + 64e6                         # room for about one large job at a time
    srv = Server(workers=4, budget_bytes=budget, bytes_per_point=4000.0, small_job=10_000,
                 batch_points=60_000, keep_results=False)
    srv.run(jobs)
    assert srv.peak_reserved <= budget


def test_large_job_in_the_mix_matches_oracle():
    """A 1.5M-point clustered 3D job served among smaller ones that arrive
    while it runs equals the oracle's DT of that job, element by element."""
    from paper_1902_07554_gb300.serve import Job, Server
    big = pointsets.job_points(1_500_000, "clustered", 12345)
    jobs = [Job(0.0, 0, big)]
    sizes, kinds, seeds = pointsets.serve_jobs(10, seed=21, lo=1000, hi=100_000)
    for i in range(10):
        jobs.append(Job(0.01 * (i + 1), i + 1, pointsets.job_points(sizes[i], kinds[i], seeds[i])))
    srv = Server(workers=3)
    summary = srv.run(jobs)
    assert summary["jobs"] == 11
    res = {r.jid: r for r in srv.results()}
    assert np.array_equal(res[0].simplices.astype(np.int64), oracle.delaunay(big))
    for j in jobs[1:]:
        assert np.array_equal(res[j.jid].simplices.astype(np.int64), oracle.delaunay(j.points)), j.jid
