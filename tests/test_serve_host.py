"""Host logic of the continuous-batching server (serve.py) with stand-ins for
the library context and its stream: capacity from the budget model, every
job served exactly once with its own result, jobs finishing in the engine's
order rather than their arrival order, failed jobs reported, launches
counted.  No GPU: the stand-in stream "inserts" a fixed number of points per
run() call for every admitted job, so small jobs finish first."""
import threading
import time

import numpy as np
import pytest

from paper_1902_07554_gb300 import serve


class FakeTri:
    def __init__(self, device, **config):
        pass

    def close(self):
        pass


class FakeStream:
    """Admits queued jobs while they fit in `capacity` points, then advances
    every admitted job by `per_run` points per run(); rows name their job."""
    per_run = 5000

    def __init__(self, tri, dim, capacity, max_jobs=256):
        self.dim, self.capacity, self.max_jobs = dim, capacity, max_jobs
        self.lock = threading.Lock()
        self.jobs = {}        # id -> dict(points, left, status)
        self.queue = []
        self.next = 1
        self.quanta = 0
        self.used = 0

    def submit(self, points):
        with self.lock:
            jid = self.next
            self.next += 1
            bad = not np.all(np.isfinite(points))
            self.jobs[jid] = dict(points=points, left=len(points), status=-1 if bad else 0)
            if not bad:
                self.queue.append(jid)
            return jid

    def run(self, quanta=1):
        time.sleep(0.001)                  # one engine pass takes time
        with self.lock:
            for jid in list(self.queue):
                j = self.jobs[jid]
                running = sum(1 for x in self.jobs.values() if x["status"] == 1)
                if self.used + len(j["points"]) <= self.capacity and running < self.max_jobs:
                    j["status"] = 1
                    self.used += len(j["points"])
                    self.queue.remove(jid)
            for j in self.jobs.values():
                if j["status"] == 1:
                    j["left"] -= self.per_run
                    if j["left"] <= 0:
                        j["status"] = 2
                        self.used -= len(j["points"])
            self.quanta += 1
            return len(self.queue) + sum(1 for x in self.jobs.values() if x["status"] == 1)

    def status(self, jid):
        with self.lock:
            return self.jobs[jid]["status"], 0

    def fetch(self, jid):
        with self.lock:
            P = self.jobs[jid]["points"]
            return np.full((len(P), 1), P[0, 0])

    def release(self, jid):
        with self.lock:
            del self.jobs[jid]

    def info(self):
        with self.lock:
            return {"capacity": self.capacity, "free_points": self.capacity - self.used, "device_bytes": 1000,
                    "queued": len(self.queue), "running": 0, "quanta": self.quanta, "rounds": 10 * self.quanta,
                    "launches": 80 * self.quanta}

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(serve, "Triangulator", FakeTri)
    monkeypatch.setattr(serve, "Stream", FakeStream)


def _jobs(sizes, gap=0.0):
    # the first coordinate of every point is the job id, so results name their job
    return [serve.Job(i * gap, i, np.full((n, 2), float(i))) for i, n in enumerate(sizes)]


def test_capacity_from_the_budget_model(fake):
    srv = serve.Server(budget_bytes=1e9 + 2000 * 50_000, model=(1e9, 2000.0))
    assert srv.capacity == 50_000
    srv = serve.Server(budget_bytes=1e15, model=(1e9, 2000.0))
    assert srv.capacity == 1 << 25                       # the stream's own limit


def test_every_job_served_once_with_its_own_result(fake):
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in rng.integers(100, 60_000, size=40)]
    srv = serve.Server(model=(0.0, 1.0), capacity=200_000)
    s = srv.run(_jobs(sizes, gap=0.0005))
    res = srv.results()
    assert [r.jid for r in res] == list(range(40)) and s["jobs"] == 40 and s["failed"] == 0
    for r in res:
        assert r.n == sizes[r.jid] and np.all(r.simplices == r.jid) and r.done >= r.arrival
    assert s["peak_running_points"] <= 200_000 and s["launches"] > 0 and s["quanta"] > 0
    assert s["p99_ms"] >= s["p50_ms"] > 0 and s["rows_out"] == sum(sizes)


def test_small_jobs_overtake_a_large_one(fake):
    """A large job admitted first does not hold back small ones that arrive
    after it: they finish in fewer engine passes."""
    sizes = [150_000] + [2_000] * 8
    srv = serve.Server(model=(0.0, 1.0), capacity=400_000)
    srv.run(_jobs(sizes, gap=0.001))
    res = {r.jid: r for r in srv.results()}
    assert all(res[i].done < res[0].done for i in range(1, 9))


def test_failed_jobs_are_reported(fake):
    jobs = _jobs([1000, 2000, 3000])
    jobs[1].points[5, 0] = np.nan
    srv = serve.Server(model=(0.0, 1.0), capacity=100_000)
    s = srv.run(jobs)
    res = {r.jid: r for r in srv.results()}
    assert s["failed"] == 1 and res[1].status == -1 and res[1].simplices is None
    assert res[0].status == 2 and res[2].status == 2


def test_k_for_and_arrivals():
    assert serve.k_for(1000) == 1 and serve.k_for(10_000_000) == 1
    assert serve.k_for(10_000_000, divide=True) == 64 and serve.k_for(200_000, divide=True) == 4
    a = serve.poisson_arrivals(2000, 50.0, 1)
    assert np.all(np.diff(a) > 0) and abs(a[-1] / 2000 - 1 / 50.0) < 0.005
