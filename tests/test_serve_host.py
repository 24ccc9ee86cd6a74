"""Host logic of the continuous-batching server (serve.py) with a stand-in
for the library context: admission under the memory budget, packing of small
jobs into batched calls, every job served exactly once with its own result.
No GPU: the stand-in returns one row per point and records what it ran."""
import threading
import time

import numpy as np

from paper_1902_07554_gb300 import serve


class FakeTri:
    """Stands in for Triangulator: records calls, returns rows that name their job."""
    calls = []
    lock = threading.Lock()

    def __init__(self, device, **config):
        self._launches = 0

    def triangulate(self, P, k=1, sample_frac=0.0, fetch=True):
        time.sleep(0.002)
        with FakeTri.lock:
            FakeTri.calls.append(("single", [len(P)]))
        return np.full((len(P), 1), P[0, 0], dtype=np.float64)

    def triangulate_batch(self, P, off):
        time.sleep(0.002)
        sizes = [int(off[i + 1] - off[i]) for i in range(len(off) - 1)]
        with FakeTri.lock:
            FakeTri.calls.append(("batch", sizes))
        return [np.full((s, 1), P[off[i], 0], dtype=np.float64) for i, s in enumerate(sizes)]

    def stats(self):
        class S:
            launches = 3
        return S()

    def close(self):
        pass


def _jobs(sizes, gap=0.0):
    # the first coordinate of every point is the job id, so results name their job
    return [serve.Job(i * gap, i, np.full((n, 2), float(i))) for i, n in enumerate(sizes)]


def test_every_job_served_once_with_its_own_result(monkeypatch):
    monkeypatch.setattr(serve, "Triangulator", FakeTri)
    FakeTri.calls = []
    rng = np.random.default_rng(3)
    sizes = [int(x) for x in rng.integers(100, 200_000, size=60)]
    srv = serve.Server(workers=3, budget_bytes=1e12, bytes_per_point=100.0, small_job=65_536,
                       batch_points=300_000)
    out = srv.run(_jobs(sizes, gap=0.0005))
    res = srv.results()
    assert [r.jid for r in res] == list(range(60))
    for r in res:
        assert r.n == sizes[r.jid] and len(r.simplices) == sizes[r.jid]
        assert np.all(r.simplices == r.jid) and r.done >= r.start >= 0
        assert r.batched == (sizes[r.jid] <= 65_536)
    assert out["jobs"] == 60 and out["points"] == sum(sizes) and out["rows_out"] == sum(sizes)
    assert out["launches"] == 3 * len(FakeTri.calls)
    for kind, s in FakeTri.calls:
        if kind == "batch":
            assert all(x <= 65_536 for x in s) and sum(s) <= 300_000
        else:
            assert s[0] > 65_536


def test_admission_keeps_the_reservation_within_the_budget(monkeypatch):
    monkeypatch.setattr(serve, "Triangulator", FakeTri)
    FakeTri.calls = []
    bpp = 1000.0
    sizes = [150_000] * 8 + [20_000] * 20
    budget = 2 * (bpp * 150_000 + 64e6) + 1.0      # room for two large jobs at a time
    srv = serve.Server(workers=4, budget_bytes=budget, bytes_per_point=bpp)
    out = srv.run(_jobs(sizes), realtime=False)
    assert out["jobs"] == len(sizes)
    assert srv.peak_reserved <= budget
    assert srv._reserved == 0.0


def test_a_job_larger_than_the_budget_still_runs_alone(monkeypatch):
    monkeypatch.setattr(serve, "Triangulator", FakeTri)
    FakeTri.calls = []
    srv = serve.Server(workers=2, budget_bytes=1e6, bytes_per_point=1000.0)
    out = srv.run(_jobs([100_000, 100]), realtime=False)
    assert out["jobs"] == 2
    assert ("single", [100_000]) in FakeTri.calls


def test_k_for_and_arrivals():
    assert serve.k_for(10_000_000) == 1
    assert serve.k_for(100_000, divide=True) == 1
    assert serve.k_for(1_000_000, divide=True) == 16 and serve.k_for(10_000_000, divide=True) == 64
    a = serve.poisson_arrivals(20_000, 50.0, 1)
    assert np.all(np.diff(a) > 0) and abs(np.diff(a).mean() - 0.02) < 0.001
