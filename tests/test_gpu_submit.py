"""Asynchronous jobs through the C ABI (dt_submit, dt_poll,
dt_get_job_simplices, dt_release_job): every job's result equals the
oracle's DT element by element (integer output: bit-exact), jobs run while
the context serves its own calls, and errors come back through dt_poll."""
import time

import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tri():
    from paper_1902_07554_gb300 import Triangulator
    t = Triangulator(0)
    yield t
    t.close()


def _wait(tri, job, limit_s=120.0):
    t0 = time.time()
    while not tri.poll(job):
        assert time.time() - t0 < limit_s, "job did not finish"
        time.sleep(0.002)


def test_jobs_match_oracle_beside_the_contexts_own_calls(tri):
    sets = [(pointsets.uniform(6000, 2, 1), 4, 0.02), (pointsets.uniform(3000, 3, 2), 1, 0.0),
            (pointsets.clustered(4000, 3), 2, 0.05)]
    jobs = [tri.submit(P, k=k, sample_frac=f) for P, k, f in sets]
    assert jobs == sorted(jobs) and len(set(jobs)) == 3
    Q = pointsets.uniform(5000, 2, 9)                     # the context's own call, meanwhile
    assert np.array_equal(tri.triangulate(Q).astype(np.int64), oracle.delaunay(Q))
    for j, (P, _, _) in zip(jobs, sets):
        _wait(tri, j)
        assert np.array_equal(tri.job_simplices(j).astype(np.int64), oracle.delaunay(P))


def test_job_errors(tri):
    from paper_1902_07554_gb300 import DTError
    P = pointsets.uniform(1000, 2, 3)
    P[5] = P[7]
    j = tri.submit(P)
    with pytest.raises(DTError, match="DUPLICATE"):
        _wait(tri, j)
    tri.release_job(j)
    with pytest.raises(DTError, match="ARG"):
        tri.poll(j)
    with pytest.raises(DTError, match="ARG"):
        tri.submit(np.zeros((2, 3)))
    with pytest.raises(DTError, match="ARG"):
        tri.poll(10 ** 9)
    ok = tri.submit(pointsets.uniform(500, 3, 4))
    _wait(tri, ok)
    assert tri.job_simplices(ok, release=False).shape[1] == 4
    tri.release_job(ok)
