"""Continuous-batching server for triangulation jobs on one GPU.

Jobs (point sets) arrive over time.  A job is admitted when a worker is free
and its estimated device memory fits the remaining budget; small jobs that are
waiting together are packed into one batched call (dt_triangulate_batch),
large ones run the divide-and-conquer path.  Every worker owns a library
context with its own CUDA stream, so admitted work from different workers
overlaps on the device while new requests keep arriving.  Latency is measured
from a job's arrival to the moment its simplices are back on the host.

Everything runs through the library's C ABI; Python only schedules.
"""
from __future__ import annotations

import heapq
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Triangulator


@dataclass(order=True)
class Job:
    arrival: float
    jid: int = field(compare=False)
    points: np.ndarray = field(compare=False, repr=False)
    k: int = field(compare=False, default=1)
    frac: float = field(compare=False, default=0.005)


@dataclass
class Result:
    jid: int
    n: int
    arrival: float
    start: float
    done: float
    simplices: np.ndarray | None
    worker: int
    batched: bool


class Server:
    """Admission, batching and execution of jobs on `workers` contexts.

    bytes_per_point: device-memory model of one job (measured once from the
    library's pool after a run of the target shape; see calibrate()).
    """

    def __init__(self, device: int = 0, workers: int = 3, budget_bytes: float = 120e9,
                 bytes_per_point: float = 6000.0, small_job: int = 65_536, batch_points: int = 2_000_000,
                 keep_results: bool = True, **config):
        self.device = device
        self.workers = workers
        self.budget = float(budget_bytes)
        self.bpp = float(bytes_per_point)
        self.small_job = small_job
        self.batch_points = batch_points
        self.keep = keep_results
        self.config = config
        self._lock = threading.Condition()
        self._queue: list[Job] = []            # arrived, not yet admitted (by arrival time)
        self._reserved = 0.0
        self._results: list[Result] = []
        self._rows_out = 0                      # simplices copied back to the host
        self._launches = 0                      # CUDA kernels launched by the library
        self._closed = False
        self._t0 = None
        self.peak_reserved = 0.0

    # ------------------------------------------------------------------ model
    def estimate(self, n: int) -> float:
        return self.bpp * n + 64e6

    # ------------------------------------------------------------------ clients
    def submit(self, job: Job):
        with self._lock:
            heapq.heappush(self._queue, job)
            self._lock.notify_all()

    def close(self):
        with self._lock:
            self._closed = True
            self._lock.notify_all()

    def now(self) -> float:
        return time.perf_counter() - self._t0

    # ------------------------------------------------------------------ scheduling
    def _take(self):
        """Next work unit for a free worker: one large job, or a pack of the
        small jobs waiting now, limited by the memory budget.  None = wait."""
        if not self._queue:
            return None
        head = self._queue[0]
        n = len(head.points)
        if n > self.small_job:
            need = self.estimate(n)
            if self._reserved + need > self.budget and self._reserved > 0:
                return None
            heapq.heappop(self._queue)
            self._reserved += need
            return [head], need
        pack, total, need = [], 0, 0.0
        rest = []
        while self._queue:
            j = heapq.heappop(self._queue)
            m = len(j.points)
            e = self.estimate(m)
            if m <= self.small_job and total + m <= self.batch_points and \
                    (self._reserved + need + e <= self.budget or not pack and self._reserved == 0):
                pack.append(j)
                total += m
                need += e
            else:
                rest.append(j)
        for j in rest:
            heapq.heappush(self._queue, j)
        if not pack:
            return None
        self._reserved += need
        return pack, need

    def _worker(self, w: int):
        tri = Triangulator(self.device, **self.config)
        try:
            while True:
                with self._lock:
                    while True:
                        unit = self._take()
                        if unit is not None:
                            break
                        if self._closed and not self._queue:
                            return
                        self._lock.wait(timeout=0.005)
                    self.peak_reserved = max(self.peak_reserved, self._reserved)
                jobs, need = unit
                start = self.now()
                if len(jobs) == 1 and len(jobs[0].points) > self.small_job:
                    j = jobs[0]
                    out = tri.triangulate(j.points, k=j.k, sample_frac=j.frac, fetch=True)
                    outs, batched = [out], False
                else:
                    P = np.concatenate([j.points for j in jobs]) if len(jobs) > 1 else jobs[0].points
                    off = np.zeros(len(jobs) + 1, dtype=np.int64)
                    off[1:] = np.cumsum([len(j.points) for j in jobs])
                    outs, batched = tri.triangulate_batch(P, off), True
                done = self.now()
                launched = tri.stats().launches
                with self._lock:
                    self._reserved -= need
                    self._rows_out += sum(len(o) for o in outs)
                    self._launches += launched
                    for j, o in zip(jobs, outs):
                        self._results.append(Result(j.jid, len(j.points), j.arrival, start, done,
                                                    o if self.keep else None, w, batched))
                    self._lock.notify_all()
        finally:
            tri.close()

    # ------------------------------------------------------------------ driver
    def run(self, jobs: list[Job], realtime: bool = True) -> dict:
        """Replays `jobs` (arrival times in seconds from start) and serves them."""
        self._t0 = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(w,), daemon=True) for w in range(self.workers)]
        for t in threads:
            t.start()
        for j in sorted(jobs, key=lambda j: j.arrival):
            if realtime:
                delay = j.arrival - self.now()
                if delay > 0:
                    time.sleep(delay)
            self.submit(j)
        self.close()
        for t in threads:
            t.join()
        return self.summary()

    def results(self) -> list[Result]:
        return sorted(self._results, key=lambda r: r.jid)

    def summary(self) -> dict:
        res = self._results
        if not res:
            return {}
        lat = np.array([r.done - r.arrival for r in res])
        pts = sum(r.n for r in res)
        span = max(r.done for r in res) - min(r.arrival for r in res)
        return {"jobs": len(res), "points": pts, "makespan_s": span,
                "throughput_mpts": pts / span / 1e6 if span > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "batched_jobs": sum(r.batched for r in res),
                "peak_reserved_gb": self.peak_reserved / 1e9, "rows_out": self._rows_out,
                "launches": self._launches}


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def k_for(n: int, divide: bool = False) -> int:
    """Partitions for a job of n points.  On one GPU the direct insertion
    (k = 1) was faster than the divide-and-conquer path at every size measured
    (1k to 4M points: the border triangulation and the sample DT cost more
    than the smaller partial triangulations save), so jobs run directly unless
    `divide` asks for about 64k points per partition."""
    if not divide or n < 131_072:
        return 1
    return int(min(64, max(2, 2 ** round(math.log2(n / 65_536)))))
