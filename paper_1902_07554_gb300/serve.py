"""Continuous-batching server for triangulation jobs on one GPU.

Jobs (point sets) arrive over time.  The server keeps ONE resident insertion
engine (the library's stream, dt_stream_*): device buffers for `capacity`
points, sized from a device-memory budget with a per-point cost measured from
the library itself (`calibrate`).  An arriving job is queued at once; the
engine, which runs every admitted job's insertion rounds together, returns
to the host at the next round boundary, admits the queued jobs that fit into
free room, and hands back each job as soon as its last point is inserted.
Small jobs therefore never wait for a large one to finish, and all jobs in
flight share every round's launches.  Latency is measured from a job's
arrival to the moment its simplices are on the host.

Everything runs through the library's C ABI; Python only schedules.
"""
from __future__ import annotations

import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import Stream, Triangulator


@dataclass(order=True)
class Job:
    arrival: float
    jid: int = field(compare=False)
    points: np.ndarray = field(compare=False, repr=False)
    k: int = field(compare=False, default=1)          # kept for callers of the plain path; the stream inserts directly
    frac: float = field(compare=False, default=0.005)


@dataclass
class Result:
    jid: int
    n: int
    arrival: float
    start: float
    done: float
    simplices: np.ndarray | None
    status: int


def calibrate(device: int = 0, dim: int = 3, small: int = 1 << 16, large: int = 1 << 18) -> tuple[float, float]:
    """Device bytes of a stream as a + b * capacity, measured: two streams of
    `small` and `large` points are opened on `device` and their reported
    device bytes are fitted.  Returns (a, b)."""
    out = []
    for cap in (small, large):
        with Triangulator(device) as tri:
            st = Stream(tri, dim, cap, 64)
            out.append(st.info()["device_bytes"])
            st.close()
    b = (out[1] - out[0]) / (large - small)
    return out[0] - b * small, b


class Server:
    """One stream on `device`; capacity = (budget_bytes - fixed) / per point,
    from `calibrate` (or the model given), at most 2^25 points."""

    def __init__(self, device: int = 0, dim: int = 3, budget_bytes: float = 120e9, max_jobs: int = 256,
                 model: tuple[float, float] | None = None, keep_results: bool = True, capacity: int | None = None,
                 **config):
        self.device = device
        self.dim = dim
        self.budget = float(budget_bytes)
        self.model = model or calibrate(device, dim)
        fixed, per_point = self.model
        cap = int((self.budget - fixed) / per_point) if capacity is None else int(capacity)
        self.capacity = max(1 << 12, min(cap, (1 << 25)))
        self.max_jobs = max_jobs
        self.keep = keep_results
        self.config = config
        self._results: list[Result] = []
        self._rows_out = 0
        self._launches = 0
        self._lock = threading.Condition()
        self._t0 = None
        self.peak_running_points = 0
        self.info = {}

    def now(self) -> float:
        return time.perf_counter() - self._t0

    def run(self, jobs: list[Job], realtime: bool = True) -> dict:
        """Replays `jobs` (arrival times in seconds from the start): a feeder
        thread submits each job at its arrival time while this thread drives
        the engine and collects finished jobs."""
        tri = Triangulator(self.device, **self.config)
        stream = Stream(tri, self.dim, self.capacity, self.max_jobs)
        ids = {}                              # library job id -> Job
        start = {}
        submitted = [0]
        errors = []
        self._t0 = time.perf_counter()
        order = sorted(jobs, key=lambda j: j.arrival)

        def feeder():
            try:
                for j in order:
                    if realtime:
                        delay = j.arrival - self.now()
                        if delay > 0:
                            time.sleep(delay)
                    jid = stream.submit(j.points)
                    with self._lock:
                        ids[jid] = j
                        start[jid] = self.now()
                        submitted[0] += 1
                        self._lock.notify_all()
            except Exception as e:            # reported by the driver loop
                errors.append(e)
                with self._lock:
                    submitted[0] = len(order)
                    self._lock.notify_all()

        th = threading.Thread(target=feeder, daemon=True)
        th.start()
        finished: set[int] = set()
        l0 = stream.info()["launches"]
        try:
            while True:
                with self._lock:
                    open_ids = [jid for jid in ids if jid not in finished]
                    all_in = submitted[0] == len(order)
                    if not open_ids:
                        if all_in:
                            break
                        self._lock.wait(timeout=0.01)      # nothing in flight: wait for an arrival
                        continue
                stream.run(1)                              # admit, then rounds until a job ends or one arrives
                info = stream.info()
                self.peak_running_points = max(self.peak_running_points, info["capacity"] - info["free_points"])
                for jid in open_ids:
                    st, _ = stream.status(jid)
                    if st in (0, 1):
                        continue
                    rows = stream.fetch(jid) if st == 2 else None
                    t = self.now()
                    j = ids[jid]
                    self._results.append(Result(j.jid, len(j.points), j.arrival, start[jid], t,
                                                rows if self.keep else None, st))
                    if rows is not None:
                        self._rows_out += len(rows)
                    stream.release(jid)
                    finished.add(jid)
            if errors:
                raise errors[0]
        finally:
            th.join(timeout=60)
            self.info = stream.info()
            self._launches = self.info["launches"] - l0
            stream.close()
            tri.close()
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
                "mean_ms": float(lat.mean() * 1e3), "failed": sum(r.status != 2 for r in res),
                "capacity_points": self.capacity, "peak_running_points": self.peak_running_points,
                "device_gb": self.info.get("device_bytes", 0) / 1e9, "quanta": self.info.get("quanta", 0),
                "rounds": self.info.get("rounds", 0), "rows_out": self._rows_out, "launches": self._launches,
                "model_bytes_per_point": self.model[1]}


def poisson_arrivals(count: int, rate_per_s: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def k_for(n: int, divide: bool = False) -> int:
    """Partitions for a job of n points on the plain path.  On one GPU the
    direct insertion (k = 1) was faster than the divide-and-conquer path at
    every size measured (1k to 4M points: the border triangulation and the
    sample DT cost more than the smaller partial triangulations save), so
    jobs run directly unless `divide` asks for about 64k points per
    partition."""
    if not divide or n < 131_072:
        return 1
    return int(min(64, max(2, 2 ** round(math.log2(n / 65_536)))))
