"""GB300 sample-based divide-and-conquer Delaunay triangulation.

A thin ctypes binding over the C ABI in include/dt.h.  Every step of the
triangulation runs in the CUDA library ``_build/libgb300dt.so``; this module
only marshals arguments.  There is no CPU fallback: if the library is missing
or no CUDA device is visible, the calls raise.

Typical use::

    from paper_1902_07554_gb300 import Triangulator
    with Triangulator() as tri:
        simplices = tri.triangulate(points, k=16, sample_frac=0.005)
        stats = tri.stats()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["Triangulator", "Stream", "DTError", "load_library", "declared_symbols", "Config", "Stats",
           "DIVIDE_SAMPLE", "DIVIDE_KD", "PRIM_GRID", "PRIM_BBOX", "PRIM_POINTS", "INITS"]

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "dt.h")

DIVIDE_SAMPLE, DIVIDE_KD = 0, 1
PRIM_GRID, PRIM_BBOX, PRIM_POINTS = 0, 1, 2
WEIGHTS = {"log": 0, "constant": 1, "inverse": 2, "linear": 3}
INITS = {"auto": 0, "hilbert": 1, "kd": 2}

ERRORS = {-1: "DT_E_ARG", -2: "DT_E_DUPLICATE", -3: "DT_E_DEGENERATE", -4: "DT_E_NOMEM",
          -5: "DT_E_TIMEOUT", -6: "DT_E_OVERFLOW", -7: "DT_E_CUDA", -8: "DT_E_RANGE",
          -9: "DT_E_INTERNAL"}


class DTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("divide", ctypes.c_int), ("primitive", ctypes.c_int), ("weight", ctypes.c_int),
                ("lp_rounds", ctypes.c_int), ("epsilon", ctypes.c_double),
                ("grid_cell", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("base_threshold", ctypes.c_int), ("validate", ctypes.c_int),
                ("cavity_cap", ctypes.c_int), ("profile", ctypes.c_int), ("neighbors", ctypes.c_int),
                ("first_batch", ctypes.c_int), ("brio_growth", ctypes.c_int),
                ("small_rounds", ctypes.c_int), ("brio_drain", ctypes.c_int),
                ("partition_init", ctypes.c_int), ("recursive", ctypes.c_int),
                ("active_ratio", ctypes.c_int), ("nominate_rings", ctypes.c_int), ("partitioner", ctypes.c_int),
                ("round_limit", ctypes.c_int), ("walk_limit", ctypes.c_int), ("arena_factor", ctypes.c_int),
                ("cavity_blocks", ctypes.c_int), ("cavity_occupancy", ctypes.c_int),
                ("cavity_group", ctypes.c_int)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("simplices", ctypes.c_int64), ("k", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("eta", ctypes.c_int64),
                ("border_vertices", ctypes.c_int64), ("border_simplices", ctypes.c_int64),
                ("border_dt_simplices", ctypes.c_int64), ("imbalance", ctypes.c_double),
                ("cv", ctypes.c_double), ("o_dt", ctypes.c_double), ("cut_weight", ctypes.c_int64),
                ("rounds_max", ctypes.c_int32), ("exact_calls", ctypes.c_int32),
                ("ms_total", ctypes.c_double), ("ms_phase", ctypes.c_double * 8),
                ("partition_size_max", ctypes.c_int64), ("partition_size_min", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("hull_facets", ctypes.c_int64), ("validated", ctypes.c_int32),
                ("reserved_i", ctypes.c_int32)]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "ms_phase" else v
        return d


class StreamInfo(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_int64), ("free_points", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("running", ctypes.c_int32), ("queued", ctypes.c_int32), ("quanta", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Validation(ctypes.Structure):
    """Result of the Delaunay certificate (dt_validate)."""
    _fields_ = [(name, ctypes.c_int64) for name in (
        "simplices", "interior_facets", "hull_facets", "edges", "euler", "bad_index", "flat", "non_manifold",
        "asymmetric", "folded", "non_delaunay", "non_convex", "unused_points", "pivot_limit", "violations")]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def declared_symbols() -> list[str]:
    """Names of the entry points declared in include/dt.h."""
    import re
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^DT_API\s+[\w\s\*]+?\b(dt_\w+)\s*\(", txt, flags=re.M)))


def load_library(build: bool = True):
    """Load (building first if needed) the CUDA library; raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    L = ctypes.CDLL(path)
    p, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "dt_config_default": ([p], i32),
        "dt_create": ([p, i32, p, p], i32),
        "dt_set_config": ([p, p], i32),
        "dt_triangulate": ([p, p, i64, i32, i32, dbl], i32),
        "dt_get_simplices": ([p, p, i64, p], i32),
        "dt_get_simplices_device": ([p, p, p], i32),
        "dt_get_stats": ([p, p], i32),
        "dt_get_labels": ([p, p, i64], i32),
        "dt_get_sample": ([p, p, i64, p], i32),
        "dt_get_sample_blocks": ([p, p, i64], i32),
        "dt_get_border_vertices": ([p, p, i64, p], i32),
        "dt_last_error": ([p], ctypes.c_char_p),
        "dt_destroy": ([p], None),
        "dt_eval_predicates": ([p, p, i64, i32, p, i32, p, i64, p], i32),
        "dt_label_points": ([p, p, i64, i32, p, p, p, i64, p], i32),
        "dt_partition_graph": ([p, p, i64, i32, p, p, i64, i32, dbl, i32, p], i32),
        "dt_get_kernel_profile": ([p, p, i32, p], i32),
        "dt_triangulate_batch": ([p, p, p, i32, i32], i32),
        "dt_get_batch_simplices": ([p, p, i64, p, p], i32),
        "dt_get_batch_status": ([p, p, i32], i32),
        "dt_select_sample_noalloc": ([i32, p, i64, i64, ctypes.c_uint64, p], i32),
        "dt_measure_fma_rate": ([i32, i32, i32, p], i32),
        "dt_stream_open": ([p, i32, i64, i32], i32),
        "dt_stream_submit": ([p, p, i64, p], i32),
        "dt_stream_run": ([p, i32, p], i32),
        "dt_stream_job": ([p, ctypes.c_uint64, p, p], i32),
        "dt_stream_fetch": ([p, ctypes.c_uint64, p, i64, p], i32),
        "dt_stream_release": ([p, ctypes.c_uint64], i32),
        "dt_stream_get_info": ([p, p], i32),
        "dt_stream_close": ([p], i32),
        "dt_get_neighbors": ([p, p, i64, p], i32),
        "dt_validate": ([p, p, i64, i32, p, i64, p], i32),
        "dt_submit": ([p, p, i64, i32, i32, dbl, p], i32),
        "dt_poll": ([p, ctypes.c_uint64, p], i32),
        "dt_get_job_simplices": ([p, ctypes.c_uint64, p, i64, p], i32),
        "dt_release_job": ([p, ctypes.c_uint64], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def fma_rate(device: int = 0, precision: int = 64, reps: int = 5) -> float:
    """Measured FP32 or FP64 FMA throughput of the device (TFLOP/s)."""
    L = load_library()
    out = ctypes.c_double(0.0)
    rc = L.dt_measure_fma_rate(device, precision, reps, ctypes.byref(out))
    if rc:
        raise DTError(rc, "dt_measure_fma_rate failed")
    return out.value


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _as_points(points):
    if hasattr(points, "data_ptr"):           # torch tensor (host or cuda)
        t = points.contiguous()
        if t.dtype != __import__("torch").float64:
            raise TypeError("points must be float64")
        return t, t.shape[0], t.shape[1]
    a = np.ascontiguousarray(points, dtype=np.float64)
    if a.ndim != 2:
        raise ValueError("points must be (n, dim)")
    return a, a.shape[0], a.shape[1]


class Triangulator:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, stream=None, **config):
        self.L = load_library()
        self.ctx = ctypes.c_void_p()
        cfg = self.default_config()
        for k, v in config.items():
            if k == "weight" and isinstance(v, str):
                v = WEIGHTS[v]
            if k == "partition_init" and isinstance(v, str):
                v = INITS[v]
            setattr(cfg, k, v)
        self._cfg = cfg
        self._job_dim = {}
        rc = self.L.dt_create(ctypes.byref(self.ctx), device, stream, ctypes.byref(cfg))
        if rc:
            raise DTError(rc, "dt_create failed (no CUDA device?)")

    def default_config(self) -> Config:
        cfg = Config()
        self.L.dt_config_default(ctypes.byref(cfg))
        return cfg

    def configure(self, **config):
        for k, v in config.items():
            if k == "weight" and isinstance(v, str):
                v = WEIGHTS[v]
            if k == "partition_init" and isinstance(v, str):
                v = INITS[v]
            setattr(self._cfg, k, v)
        self._check(self.L.dt_set_config(self.ctx, ctypes.byref(self._cfg)))

    def _check(self, rc):
        if rc:
            raise DTError(rc, self.L.dt_last_error(self.ctx).decode())

    def close(self):
        if self.ctx:
            self.L.dt_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- main call
    def triangulate(self, points, k: int = 1, sample_frac: float = 0.0, fetch: bool = True):
        """DT(points): (m, dim+1) int32 array of input indices, rows sorted."""
        P, n, dim = _as_points(points)
        self._check(self.L.dt_triangulate(self.ctx, _ptr(P), n, dim, k, float(sample_frac)))
        return self.simplices() if fetch else None

    def submit(self, points, k: int = 1, sample_frac: float = 0.0) -> int:
        """Queue DT(points) on the context's job worker; returns the job id
        (the points are copied before this returns)."""
        P, n, dim = _as_points(points)
        job = ctypes.c_uint64()
        self._check(self.L.dt_submit(self.ctx, _ptr(P), n, dim, k, float(sample_frac), ctypes.byref(job)))
        self._job_dim[job.value] = dim
        return job.value

    def poll(self, job: int) -> bool:
        """True once the job has finished; raises DTError if it failed."""
        done = ctypes.c_int()
        self._check(self.L.dt_poll(self.ctx, job, ctypes.byref(done)))
        return bool(done.value)

    def job_simplices(self, job: int, release: bool = True):
        """A finished job's simplices ((m, dim+1) int32, as triangulate
        returns); the job is released afterwards unless release is False."""
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_job_simplices(self.ctx, job, None, 0, ctypes.byref(cnt)))
        out = np.empty((cnt.value, self._job_dim[job] + 1), dtype=np.int32)
        self._check(self.L.dt_get_job_simplices(self.ctx, job, _ptr(out), cnt.value, ctypes.byref(cnt)))
        if release:
            self.release_job(job)
        return out

    def release_job(self, job: int):
        self._check(self.L.dt_release_job(self.ctx, job))
        self._job_dim.pop(job, None)

    def triangulate_batch(self, points, offsets, fetch: bool = True):
        """Independent DTs of points[offsets[i]:offsets[i+1]]; returns a list of
        (m_i, dim+1) int32 arrays of instance-local indices (or None)."""
        P, n, dim = _as_points(points)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._last_batch = len(off) - 1
        self._check(self.L.dt_triangulate_batch(self.ctx, _ptr(P), _ptr(off), len(off) - 1, dim))
        return self.batch_simplices() if fetch else None

    def batch_simplices(self):
        total = ctypes.c_int64()
        cnt = self.stats()
        nb = self._batch_count()
        ro = np.empty(nb + 1, dtype=np.int64)
        self._check(self.L.dt_get_batch_simplices(self.ctx, None, 0, _ptr(ro), ctypes.byref(total)))
        out = np.empty((total.value, cnt.dim + 1), dtype=np.int32)
        self._check(self.L.dt_get_batch_simplices(self.ctx, _ptr(out), total.value, _ptr(ro), ctypes.byref(total)))
        return [out[ro[i]:ro[i + 1]] for i in range(nb)]

    def _batch_count(self):
        # probe the last batch's instance count through the status call
        for guess in (self._last_batch,) if getattr(self, "_last_batch", None) else ():
            return guess
        raise RuntimeError("no batch")

    def batch_status(self, count):
        out = np.empty(count, dtype=np.int32)
        self._check(self.L.dt_get_batch_status(self.ctx, _ptr(out), count))
        return out

    def simplices(self, out=None):
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_simplices(self.ctx, None, 0, ctypes.byref(cnt)))
        s = self.stats()
        if out is None:
            out = np.empty((cnt.value, s.dim + 1), dtype=np.int32)
        self._check(self.L.dt_get_simplices(self.ctx, _ptr(out), cnt.value, ctypes.byref(cnt)))
        return out

    def neighbors(self, out=None):
        """Neighbour array of the last result (the merge's neighbourhood
        update): row r, column j = the simplex opposite vertex j of simplex r,
        -1 on the convex hull; rows in the order of simplices()."""
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_neighbors(self.ctx, None, 0, ctypes.byref(cnt)))
        if out is None:
            out = np.empty((cnt.value, self.stats().dim + 1), dtype=np.int32)
        self._check(self.L.dt_get_neighbors(self.ctx, _ptr(out), cnt.value, ctypes.byref(cnt)))
        return out

    def validate(self, points, simplices) -> dict:
        """Certificate that `simplices` is the Delaunay triangulation of
        `points` (see Validation); returns the counters as a dict."""
        P, n, dim = _as_points(points)
        S = simplices
        if not hasattr(S, "data_ptr"):
            S = np.ascontiguousarray(S, dtype=np.int32).reshape(-1, dim + 1)
        v = Validation()
        self._check(self.L.dt_validate(self.ctx, _ptr(P), n, dim, _ptr(S), len(S), ctypes.byref(v)))
        return v.as_dict()

    def simplex_count(self) -> int:
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_simplices(self.ctx, None, 0, ctypes.byref(cnt)))
        return cnt.value

    def stats(self) -> Stats:
        s = Stats()
        self._check(self.L.dt_get_stats(self.ctx, ctypes.byref(s)))
        return s

    def kernel_profile(self):
        cnt = ctypes.c_int()
        self._check(self.L.dt_get_kernel_profile(self.ctx, None, 0, ctypes.byref(cnt)))
        arr = (KernelProfile * max(cnt.value, 1))()
        self._check(self.L.dt_get_kernel_profile(self.ctx, arr, cnt.value, ctypes.byref(cnt)))
        return [dict(name=a.name.decode(), launches=a.launches, ms=a.ms, bytes=a.bytes, flops=a.flops)
                for a in arr[:cnt.value]]

    def labels(self):
        n = self.stats().n
        out = np.empty(n, dtype=np.int32)
        self._check(self.L.dt_get_labels(self.ctx, _ptr(out), n))
        return out

    def sample(self):
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_sample(self.ctx, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.int32)
        self._check(self.L.dt_get_sample(self.ctx, _ptr(out), cnt.value, ctypes.byref(cnt)))
        return out

    def sample_blocks(self):
        eta = len(self.sample())
        out = np.empty(eta, dtype=np.int32)
        self._check(self.L.dt_get_sample_blocks(self.ctx, _ptr(out), eta))
        return out

    def border_vertices(self):
        cnt = ctypes.c_int64()
        self._check(self.L.dt_get_border_vertices(self.ctx, None, 0, ctypes.byref(cnt)))
        out = np.empty(cnt.value, dtype=np.int32)
        self._check(self.L.dt_get_border_vertices(self.ctx, _ptr(out), cnt.value, ctypes.byref(cnt)))
        return out

    # ------------------------------------------------------------- steps
    def eval_predicates(self, points, kind: str, tuples, gid=None):
        code = {"orient": 0, "insphere": 1, "insphere_raw": 2, "closer": 3}[kind]
        P = np.ascontiguousarray(points, dtype=np.float64)
        T = np.ascontiguousarray(tuples, dtype=np.int32)
        g = None if gid is None else np.ascontiguousarray(gid, dtype=np.int64)
        out = np.empty(len(T), dtype=np.int8)
        self._check(self.L.dt_eval_predicates(self.ctx, _ptr(P), P.shape[0], P.shape[1], _ptr(g), code,
                                              _ptr(T), len(T), _ptr(out)))
        return out

    def label_points(self, P, S, srank, block):
        P = np.ascontiguousarray(P, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.float64)
        r = np.ascontiguousarray(srank, dtype=np.int64)
        b = np.ascontiguousarray(block, dtype=np.int32)
        out = np.empty(len(P), dtype=np.int32)
        self._check(self.L.dt_label_points(self.ctx, _ptr(P), len(P), P.shape[1], _ptr(S), _ptr(r), _ptr(b),
                                           len(S), _ptr(out)))
        return out

    def partition_graph(self, S, E, w, k, eps=0.05, rounds=16):
        S = np.ascontiguousarray(S, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int64)
        out = np.empty(len(S), dtype=np.int32)
        self._check(self.L.dt_partition_graph(self.ctx, _ptr(S), len(S), S.shape[1], _ptr(E), _ptr(w), len(E),
                                              k, float(eps), rounds, _ptr(out)))
        return out


class Stream:
    """Continuous batching on one context (dt_stream_*): jobs are submitted
    from any thread and join the resident engine at the next round boundary;
    one driver thread calls run().  Argument marshalling only."""

    def __init__(self, tri: "Triangulator", dim: int, capacity: int, max_jobs: int = 256):
        self.tri = tri
        self.L = tri.L
        self.dim = dim
        tri._check(self.L.dt_stream_open(tri.ctx, dim, int(capacity), int(max_jobs)))

    def submit(self, points) -> int:
        a = np.ascontiguousarray(points, dtype=np.float64)
        if a.ndim != 2 or a.shape[1] != self.dim:
            raise ValueError(f"points must be (n, {self.dim})")
        job = ctypes.c_uint64()
        rc = self.L.dt_stream_submit(self.tri.ctx, _ptr(a), len(a), ctypes.byref(job))
        if rc:
            raise DTError(rc, "dt_stream_submit")
        return job.value

    def run(self, quanta: int = 1) -> int:
        pending = ctypes.c_int()
        self.tri._check(self.L.dt_stream_run(self.tri.ctx, quanta, ctypes.byref(pending)))
        return pending.value

    def status(self, job: int):
        st, cnt = ctypes.c_int(), ctypes.c_int64()
        rc = self.L.dt_stream_job(self.tri.ctx, job, ctypes.byref(st), ctypes.byref(cnt))
        if rc:
            raise DTError(rc, "dt_stream_job")
        return st.value, cnt.value

    def fetch(self, job: int) -> np.ndarray:
        cnt = ctypes.c_int64()
        rc = self.L.dt_stream_fetch(self.tri.ctx, job, None, 0, ctypes.byref(cnt))
        if rc:
            raise DTError(rc, "dt_stream_fetch")
        out = np.empty((cnt.value, self.dim + 1), dtype=np.int32)
        rc = self.L.dt_stream_fetch(self.tri.ctx, job, _ptr(out), cnt.value, ctypes.byref(cnt))
        if rc:
            raise DTError(rc, "dt_stream_fetch")
        return out

    def release(self, job: int):
        rc = self.L.dt_stream_release(self.tri.ctx, job)
        if rc:
            raise DTError(rc, "dt_stream_release")

    def info(self) -> dict:
        out = StreamInfo()
        self.tri._check(self.L.dt_stream_get_info(self.tri.ctx, ctypes.byref(out)))
        return out.as_dict()

    def close(self):
        if self.tri.ctx:
            self.L.dt_stream_close(self.tri.ctx)

