#!/usr/bin/env python
"""Throughput and latency benchmark of the GB300 divide-and-conquer Delaunay triangulation.

Workload (default ``clustered3d_4m``): 3D, 4,000,000 float64 points (seed 3):
80 % from 50 Gaussian blobs, 20 % on a noisy heightfield; k = 64 partitions
from a 0.5 % sample (Alg. 1 + Alg. 2), grid border primitive, log edge
weights.  One step = one full dt_triangulate: divide, 64 partial
triangulations, border detection, border triangulation, hash merge,
neighbourhood update and canonical output, all on the GPU.

Printed (rank 0, one JSON line): Mpoints/s over the K timed steps (inputs
resident in HBM, L2 flushed before every step); beside it, on the same GPU
and points, the plain path (k = 1), the kd median divide (Sec. 2.3) with its
partition metrics, the 1M uniform workload as a secondary line, and a short
serving leg (Poisson arrivals of 3D jobs: p50/p99 latency of the served form
and of the plain path replayed under the same arrivals); the same metric end
to end through the C ABI from pinned host buffers (host<->device copies
inside the timed region); the roofline of the dominant kernel from the
algorithmic bytes and flops per triangulated point, with its CUDA-event time
measured live; the FP32/FP64 FMA roofs measured live; the CPU oracle timed on
a bounded sample; and the SM clocks seen.

``--impl reference`` times the CPU oracle instead (the only reference that
exists for this method: the paper ships no code), on a bounded sample.
Multi-GPU (torchrun): every rank triangulates its own independent point set
(replicas; no collective on the data path); value = all points / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pointsets  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
METRIC = "Mpoints/s for 3D DT on 1 GB300 vs plain path; p50/p99 latency under load"
WORKLOADS = {
    "uniform3d_1m": dict(n=1_000_000, dim=3, gen="uniform", seed=2, k=16, frac=0.005),
    "clustered3d_4m": dict(n=4_000_000, dim=3, gen="clustered", seed=3, k=64, frac=0.005),
    "uniform2d_10k": dict(n=10_000, dim=2, gen="uniform", seed=1, k=4, frac=0.01),
    # a smaller case of the same shape, for profiler captures (a few GB on the device)
    "uniform3d_200k": dict(n=200_000, dim=3, gen="uniform", seed=2, k=16, frac=0.005),
    # 4,096 independent 2D instances, 256..65,536 points each (log-uniform)
    "batch2d_4096": dict(n=0, dim=2, gen="batch", seed=4, k=1, frac=0.0),
    # Poisson arrivals of 3D jobs, 1,000..2,000,000 points, uniform or clustered
    "serve3d": dict(n=0, dim=3, gen="serve", seed=5, k=0, frac=0.005),
}


def max_over_ranks(x: float, dist, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job Mpoints/s: all ranks' points over the slowest rank's step time."""
    return world * n_per_rank / (ms_max / 1e3) / 1e6


def gen_points(w, seed_offset=0):
    if w["gen"] == "batch":
        return pointsets.batch_instances(seed=w["seed"])[0]
    if w["gen"] == "serve":
        sizes, kinds, seeds = pointsets.serve_jobs(8, seed=w["seed"])
        return pointsets.job_points(min(int(sizes[0]), 200_000), kinds[0], seeds[0])
    if w["gen"] == "uniform":
        return pointsets.uniform(w["n"], w["dim"], w["seed"] + seed_offset)
    return pointsets.clustered(w["n"], w["seed"] + seed_offset)


# Algorithmic work per triangulated point (3D, uniform; 2D in brackets):
# bytes = 24 coordinates + ~56 label/scatter + ~108 simplices written (6.77 x
# 16 B) + ~108 adjacency + ~25 border and hash = 320 B [90 B]; flops = ~20
# insphere filters x ~70 + ~30 orient filters x ~25 + the border
# circumspheres = ~2.3 kflop [0.6 kflop].  The points a step triangulates are
# n + eta + |vertices(B)| (the partitions, the sample and the border set).
ALG_BYTES_PER_POINT = {3: 320.0, 2: 90.0}
ALG_FLOPS_PER_POINT = {3: 2300.0, 2: 600.0}
# flops of one conflict test's first (FP32) stage, by dimension: determinant and both permanents
TEST_FLOPS = {3: 220.0, 2: 70.0}


def make_roofline(prof_tot: dict, prof_step_ms: list, units: int, dim: int, steps: int, peaks: dict,
                  peak_src: str, fma: dict | None = None, n: int | None = None):
    """Roofline of the kernel with the largest total time in the profiled
    steps (prof_tot: name -> {"ms", "launches", "bytes", "flops"} summed over
    `steps` steps; prof_step_ms: each profiled step's time; units: points
    triangulated per step).  achieved = ALG_BYTES_PER_POINT x units per step /
    the kernel's time per step (= the per-launch bytes over the mean launch
    time), against the measured HBM copy bandwidth.  The kernel's own count of
    the bytes it gathers is reported beside it (gather_bytes_per_launch), not
    as `achieved`.  fp64 / fp32: ALG_FLOPS_PER_POINT x units against the FMA
    rates measured live (fma: {"fp32": TF/s, "fp64": TF/s}).  traffic = the
    stored ncu DRAM bytes per input point (n points) scaled to one launch,
    when taken on the current kernel source."""
    dom = max(prof_tot.items(), key=lambda kv: kv[1]["ms"]) if prof_tot else None
    if not dom or units <= 0:
        return None
    name, a = dom
    steps = max(steps, 1)
    launches_per_step = a["launches"] / steps
    kernel_s = a["ms"] / steps / 1e3                              # kernel time per step
    alg_bytes = ALG_BYTES_PER_POINT[dim] * units                  # per step
    achieved = alg_bytes / kernel_s / 1e9 if kernel_s > 0 else 0.0
    per_launch_ms = a["ms"] / max(a["launches"], 1)
    bpp = stored_cavity_traffic() if name == "k_cavity_w<3>" else None
    traffic = bpp * (n or units) / max(launches_per_step, 1) if bpp else None
    tests = a["flops"] / TEST_FLOPS[dim] / steps
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "algorithmic": f"{ALG_BYTES_PER_POINT[dim]:.0f} B per triangulated point x {units} points "
                               f"(n + eta + |vertices(B)|) per step, over the kernel's CUDA-event time per step",
                "bytes_per_launch": alg_bytes / max(launches_per_step, 1), "ms_per_launch": per_launch_ms,
                "launches_per_step": launches_per_step,
                "gather_bytes_per_launch": a["bytes"] / max(a["launches"], 1),
                "traffic_source": ("ncu DRAM bytes per input point (uniform3d_200k, host-driven rounds) scaled to "
                                   "one launch; profiles/k_cavity_w_traffic.md") if traffic else None,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "share_of_step": a["ms"] / sum(prof_step_ms) if sum(prof_step_ms) > 0 else None,
                "timing": "CUDA events around every launch, profiled steps after the timed region",
                "conflict_tests_per_point": tests / units}
    flops = ALG_FLOPS_PER_POINT[dim] * units / kernel_s / 1e12 if kernel_s > 0 else 0.0
    for prec in ("fp64", "fp32"):
        pk = (fma or {}).get(prec)
        if pk:
            roofline[prec] = {"bound": "alu", "achieved": flops, "peak": pk, "unit": "TFLOP/s", "frac": flops / pk,
                              "peak_source": f"measured live: dt_measure_fma_rate({prec[2:]}), FMA chains on every SM",
                              "work": f"{ALG_FLOPS_PER_POINT[dim]:.0f} flops per triangulated point"}
    return roofline


def cavity_fingerprint() -> str:
    """SHA-1 of the source of the dominant kernel (region growth + k_cavity_w):
    a stored DRAM-traffic figure only applies to the kernel it was taken on."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_1902_07554_gb300", "csrc", "engine_core.cuh")).read()
    a = src.find("__device__ __forceinline__ void grow_region(")
    b = src.find("// Second growth of large region")
    return hashlib.sha1(src[a:b].encode()).hexdigest() if a >= 0 and b > a else ""


def stored_cavity_traffic():
    """DRAM bytes per input point of k_cavity_w<3> over one triangulation, from
    the ncu capture summarised in profiles/k_cavity_w_traffic.md, if that
    capture was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "k_cavity_w_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    import re
    fp = re.search(r"^fingerprint: ([0-9a-f]{40})$", txt, flags=re.M)
    bpp = re.search(r"^dram_bytes_per_point: ([0-9.eE+]+)$", txt, flags=re.M)
    if not fp or not bpp or fp.group(1) != cavity_fingerprint():
        return None
    return float(bpp.group(1))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for j, nm in enumerate(names):
                if len(r) > 5 + j and r[5 + j].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def cpu_baseline(w, budget_s: float = 15.0):
    """The CPU oracle (single-threaded C Bowyer-Watson) on a bounded sample of
    the workload: the first m points, m chosen to take roughly budget_s."""
    import oracle
    P = gen_points(w)
    m = min(w["n"], 20_000 if w["dim"] == 3 else 100_000)
    t = time.perf_counter()
    oracle.delaunay(P[:m])
    dt = time.perf_counter() - t
    # grow the sample once towards the budget
    m2 = int(min(w["n"], m * max(1.0, budget_s / max(dt, 1e-3) * 0.8)))
    if m2 > m:
        t = time.perf_counter()
        oracle.delaunay(P[:m2])
        dt = time.perf_counter() - t
        m = m2
    return {"value": m / dt / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
            "sample": f"first {m} of the {w['n']} workload points, one full DT by the C oracle, {dt:.2f} s",
            "host_cores": os.cpu_count(), "cpu_model": cpu_model()}


def cpu_model() -> str:
    """The host CPU's model name (or its architecture when /proc does not say)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_batch_chunk(job):
    """Worker of the all-core oracle baseline: generates and triangulates the
    batch instances it is given; returns their point count."""
    import oracle
    ids, count, seed = job
    pts = 0
    for i in ids:
        Q = pointsets.batch_instance(i, count=count, seed=seed)
        oracle.delaunay(Q)
        pts += len(Q)
    return pts


def cpu_baseline_batch(P, off, seed: int, budget_s: float = 8.0):
    """The CPU oracle on the batch workload's first instances: one core
    (instances in order for about budget_s), then every host core (a spawn
    pool started and warmed before the clock; each process generates and
    triangulates its share of as many instances per core)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import oracle
    count = len(off) - 1
    t0 = time.perf_counter()
    i = 0
    while i < count and (i == 0 or time.perf_counter() - t0 < budget_s):
        oracle.delaunay(P[off[i]:off[i + 1]])
        i += 1
    dt1 = time.perf_counter() - t0
    pts1 = int(off[i] - off[0])
    cores = os.cpu_count() or 1
    m = min(count, i * cores)
    shares = [(list(range(c, m, cores)), count, seed) for c in range(cores)]
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_batch_chunk, [([0], count, seed)] * cores))   # start and warm the processes
        t0 = time.perf_counter()
        ptsn = sum(ex.map(_oracle_batch_chunk, shares))
        dtn = time.perf_counter() - t0
    return {"value": pts1 / dt1 / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
            "sample": f"first {i} of the {count} instances ({pts1} points), one full DT each by the C oracle, "
                      f"one core, {dt1:.2f} s",
            "all_cores": {"value": ptsn / dtn / 1e6, "unit": "Mpoints/s", "cores": cores,
                          "sample": f"first {m} instances ({ptsn} points) spread over {cores} processes, {dtn:.2f} s"},
            "cpu_model": cpu_model()}


def cpu_baseline_jobs(pts, budget_s: float = 8.0):
    """The CPU oracle on the serving workload's first jobs, one core, in order
    for about budget_s (at least one job; every job is cut to its first
    100,000 points)."""
    import oracle
    t0 = time.perf_counter()
    done, npts = 0, 0
    while done < len(pts) and (done == 0 or time.perf_counter() - t0 < budget_s):
        Q = pts[done][:100_000]
        oracle.delaunay(Q)
        npts += len(Q)
        done += 1
    dt = time.perf_counter() - t0
    return {"value": npts / dt / 1e6, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
            "sample": f"first {done} of the {len(pts)} jobs ({npts} points; jobs cut to 100,000 points), "
                      f"one full DT each by the C oracle, {dt:.2f} s",
            "host_cores": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    P = gen_points(w)
    if w["gen"] == "batch":
        P = P[:65_536]                     # the first instances of the batch (2D)
    m = min(len(P), 60_000 if w["dim"] == 3 else 300_000)
    sample = P[:m]
    for _ in range(args.warmup):
        oracle.delaunay(sample[: m // 10])
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.delaunay(sample)
        times.append(time.perf_counter() - t)
    ms = 1e3 * sum(times) / len(times)
    value = m / (ms / 1e3) / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n": w["n"], "dim": w["dim"], "k": w["k"],
                       "sample_frac": w["frac"], "reference_sample_points": m},
            "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {m} points of the workload per step, one full DT by the C oracle"},
            "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args, w):
    """Batched form: all instances in one dt_triangulate_batch per step."""
    import torch
    from paper_1902_07554_gb300 import Triangulator
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=local)
    torch.cuda.set_stream(stream)
    P, off, kinds = pointsets.batch_instances(seed=w["seed"])
    n = int(off[-1])
    tri = Triangulator(local, stream=stream.cuda_stream)
    P_dev = torch.from_numpy(P).to(f"cuda:{local}")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")
    torch.cuda.synchronize()
    schedule = None
    if args.autotune:                      # untimed: picks the schedule the timed steps use
        from paper_1902_07554_gb300 import tune
        r = tune.autotune(tri, P_dev, offsets=off, reps=1)
        schedule = {"best": r["best"], "ms": r["ms"], "candidates": len(r["table"]),
                    "grid": {k: list(v) for k, v in tune.DEFAULT_GRID.items()}}
    for _ in range(args.warmup):
        tri.L.dt_triangulate_batch(tri.ctx, ctypes_ptr(P_dev), ctypes_ptr(off), len(off) - 1, 2)
    clk = ClockSampler(local)
    clk.start()
    step_ms, launches = [], 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = tri.L.dt_triangulate_batch(tri.ctx, ctypes_ptr(P_dev), ctypes_ptr(off), len(off) - 1, 2)
        e1.record(stream)
        e1.synchronize()
        assert rc == 0, tri.L.dt_last_error(tri.ctx)
        step_ms.append(e0.elapsed_time(e1))
        launches += tri.stats().launches
    clocks = clk.stop()
    ms = sum(step_ms) / len(step_ms)
    # end to end from pinned host memory, results back on the host
    P_pin = torch.from_numpy(P).pin_memory()
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        t = time.perf_counter()
        res = tri.triangulate_batch(P_pin, off)
        e2e.append(time.perf_counter() - t)
    nout = sum(len(r) for r in res)
    st = tri.stats()
    cpu = None if args.no_cpu_baseline else cpu_baseline_batch(P, off, w["seed"])
    line = {"metric": METRIC, "value": n / (ms / 1e3) / 1e6, "unit": "Mpoints/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "instances": len(off) - 1, "points": n, "dim": 2,
                       "l2": "flushed before every step (256 MiB write)",
                       "schedule": schedule or "default (brio_growth 150, brio_drain 8, first_batch 32, "
                                               "nominate_rings 1, cavity_blocks 16)"},
            "e2e": {"value": n / (sum(e2e) / len(e2e)) / 1e6, "unit": "Mpoints/s",
                    "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": nout * 12},
            "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu,
            "stats": {"simplices": nout, "rounds_max": st.rounds_max}}
    print(json.dumps(line), flush=True)
    return 0


def ctypes_ptr(t):
    import ctypes
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    return ctypes.c_void_p(t.ctypes.data)


def run_serving(args, w):
    """The serving workload (Poisson arrivals of 3D jobs of 1,000..2,000,000
    points, half uniform, half clustered, 120 GB budget): the served form and
    the plain path under the same arrivals at offered loads 0.5, 0.8, 0.95
    of the plain path's capacity and one overload point (1.2)."""
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    pts = serving_jobs(args.serve_jobs, seed=w["seed"])
    total = int(sum(len(p) for p in pts))
    service = plain_service_times(local, pts)
    clk = ClockSampler(local)
    clk.start()
    legs = {str(load): serving_leg(local, pts, service, load, seed=w["seed"]) for load in (0.5, 0.8, 0.95, 1.2)}
    clocks = clk.stop()
    main_leg = legs["0.8"]
    cpu = None if args.no_cpu_baseline else cpu_baseline_jobs(pts)
    line = {"metric": METRIC, "value": main_leg["served"]["throughput_mpts"], "unit": "Mpoints/s", "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": main_leg["served"]["makespan_s"] * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "jobs": len(pts), "points": total, "offered_load": 0.8,
                       "budget_gb": 120, "loads": [0.5, 0.8, 0.95, 1.2]},
            "serve": legs, "clocks": clocks, "gpu_launches": main_leg["served"].get("launches"),
            "cpu_baseline": cpu,
            "e2e": {"value": main_leg["served"]["throughput_mpts"], "unit": "Mpoints/s",
                    "h2d_bytes_per_step": total * 24, "d2h_bytes_per_step": None}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered3d_4m", choices=sorted(WORKLOADS))
    ap.add_argument("--frac", default=None,
                    help="sample size: a fraction of n, 'sqrt' (eta = sqrt n) or 'logn' (eta = log2 n); default: the "
                         "workload's")
    ap.add_argument("--weight", default=None, choices=["log", "constant", "inverse", "linear"],
                    help="edge weights of the sample graph (Table 1); default log")
    ap.add_argument("--partitioner", default="lp", choices=["lp", "ml"],
                    help="sample-graph partitioner: one level of label propagation, or multilevel")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 1M uniform secondary line")
    ap.add_argument("--no-serve-leg", action="store_true", help="skip the short serving leg")
    ap.add_argument("--serve-jobs", type=int, default=None,
                    help="jobs of the serving leg (default 40) or of the serving workload (default 400)")
    ap.add_argument("--divide", default="sample", choices=["sample", "kd"])
    ap.add_argument("--autotune", action="store_true",
                    help="time the candidate insertion schedules on the workload first and use the fastest")
    ap.add_argument("--recursive", action="store_true",
                    help="recursive bisection (log2 k bisections, k - 1 merges) instead of direct k-way")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--host-rounds", action="store_true",
                    help="drive every insertion round from the host (profile mode) in all steps, so that a "
                         "kernel profiler lists each launch; the timed value then includes the event overhead")
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.serve_jobs is None:
        args.serve_jobs = 400 if w["gen"] == "serve" else 40
    if args.impl == "reference":
        return run_reference(args, w)
    if w["gen"] == "batch":
        return run_batch(args, w)
    if w["gen"] == "serve":
        return run_serving(args, w)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_1902_07554_gb300 import Triangulator, fma_rate
    stream = torch.cuda.Stream(device=local)       # one explicit stream for torch and the library
    torch.cuda.set_stream(stream)
    # neighbors=1: the merge's neighbourhood update runs inside every step
    tri = Triangulator(local, stream=stream.cuda_stream, divide=0 if args.divide == "sample" else 1,
                       profile=1 if args.host_rounds else 0, neighbors=1, recursive=1 if args.recursive else 0)
    sample_frac = parse_frac(args.frac, w["frac"], w["n"])
    if args.weight:
        tri.configure(weight=args.weight)
    tri.configure(partitioner=1 if args.partitioner == "ml" else 0)
    P = gen_points(w, seed_offset=rank)
    n = w["n"]
    P_dev = torch.from_numpy(P).to(f"cuda:{local}")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")   # > L2 (129 MB)
    torch.cuda.synchronize()

    def steps_ms(points, k, count):
        """CUDA-event time of `count` dt_triangulate calls, L2 flushed before each."""
        out, nl = [], 0
        for _ in range(count):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tri.triangulate(points, k=k, sample_frac=sample_frac, fetch=False)
            e1.record(stream)
            e1.synchronize()
            out.append(e0.elapsed_time(e1))
            nl += tri.stats().launches
        return out, nl

    for _ in range(args.warmup):
        tri.triangulate(P_dev, k=w["k"], sample_frac=sample_frac, fetch=False)

    # ---------------- timed region: K steps on device-resident inputs (no per-kernel events)
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t0 = time.perf_counter()
    step_ms, launches = steps_ms(P_dev, w["k"], args.steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clk.stop()
    if dist:
        dist.barrier()
    ms = sum(step_ms) / len(step_ms)
    ms_max = max_over_ranks(ms, dist, f"cuda:{local}")
    value = job_value(n, world, ms_max)
    stats = tri.stats().as_dict()
    units = int(n + (stats["eta"] if stats["k"] > 1 else 0) + stats["border_vertices"])

    # ---------------- the plain path: the same points, same engine, k = 1 (no divide)
    plain_ms, _ = steps_ms(P_dev, 1, max(args.steps // 2, 3))
    plain_step = max_over_ranks(sum(plain_ms) / len(plain_ms), dist, f"cuda:{local}")
    plain = {"value": job_value(n, world, plain_step), "unit": "Mpoints/s", "ms_per_step": plain_step,
             "what": "dt_triangulate with k = 1: the same insertion engine on all points, no divide, "
                     "no border triangulation, no merge"}

    # ---------------- the other divide on the same points (sample <-> kd median, Sec. 2.3)
    other = "kd" if args.divide == "sample" else "sample"
    comparator = None
    if not args.recursive and w["k"] > 1:
        tri.configure(divide=1 if other == "kd" else 0)
        tri.triangulate(P_dev, k=w["k"], sample_frac=sample_frac, fetch=False)
        cmp_ms, _ = steps_ms(P_dev, w["k"], max(args.steps // 2, 3))
        cst = tri.stats().as_dict()
        tri.configure(divide=0 if args.divide == "sample" else 1)
        cmp_step = max_over_ranks(sum(cmp_ms) / len(cmp_ms), dist, f"cuda:{local}")
        comparator = {"divide": other, "value": job_value(n, world, cmp_step), "unit": "Mpoints/s",
                      "ms_per_step": cmp_step,
                      **{k: cst[k] for k in ("border_vertices", "border_simplices", "imbalance", "cv", "o_dt")}}

    # ---------------- the other partitioner of the sample graph (label propagation <-> multilevel)
    part_cmp = None
    if not args.recursive and w["k"] > 1 and args.divide == "sample":
        other_ml = args.partitioner != "ml"
        tri.configure(partitioner=1 if other_ml else 0)
        tri.triangulate(P_dev, k=w["k"], sample_frac=sample_frac, fetch=False)
        pm_ms, _ = steps_ms(P_dev, w["k"], max(args.steps // 2, 3))
        pst = tri.stats().as_dict()
        tri.configure(partitioner=0 if other_ml else 1)
        pm_step = max_over_ranks(sum(pm_ms) / len(pm_ms), dist, f"cuda:{local}")
        part_cmp = {"partitioner": "multilevel" if other_ml else "label propagation",
                    "value": job_value(n, world, pm_step), "unit": "Mpoints/s", "ms_per_step": pm_step,
                    "ms_partition_labels_scatter": pst["ms_phase"][1],
                    **{k: pst[k] for k in ("border_vertices", "cut_weight", "imbalance", "cv", "o_dt")}}

    # ---------------- per-kernel times: profiled steps with CUDA events around
    # every engine launch (kept out of the timed region: the events themselves
    # cost host time in the short rounds)
    tri.configure(profile=1)
    prof_tot = {}
    prof_step_ms = []
    nprof = max(1, min(args.steps, 5))
    for _ in range(nprof):
        ms1, _ = steps_ms(P_dev, w["k"], 1)
        prof_step_ms += ms1
        for kp in tri.kernel_profile():
            a = prof_tot.setdefault(kp["name"], dict(ms=0.0, launches=0, bytes=0.0, flops=0.0))
            for key in ("ms", "launches", "bytes", "flops"):
                a[key] += kp[key]
    tri.configure(profile=1 if args.host_rounds else 0)

    # ---------------- end to end: pinned host buffers through the C ABI
    P_pin = torch.from_numpy(P).pin_memory()
    nout = tri.simplex_count()
    out_pin = torch.empty((nout + 1024, w["dim"] + 1), dtype=torch.int32).pin_memory()
    e2e_ms = []
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        tri.triangulate(P_pin, k=w["k"], sample_frac=sample_frac, fetch=False)
        cnt = tri.simplex_count()
        tri.simplices(out=out_pin[:cnt])
        e2e_ms.append(1e3 * (time.perf_counter() - t))
    e2e_step = sum(e2e_ms) / len(e2e_ms)
    e2e = {"value": job_value(n, world, max_over_ranks(e2e_step, dist, f"cuda:{local}")), "unit": "Mpoints/s",
           "h2d_bytes_per_step": int(n * w["dim"] * 8), "d2h_bytes_per_step": int(cnt * (w["dim"] + 1) * 4),
           "ms_per_step": e2e_step}

    # ---------------- secondary workload (the 1M uniform configuration), fewer steps
    secondary = None
    if args.workload != "uniform3d_1m" and not args.no_secondary and w["dim"] == 3:
        w2 = WORKLOADS["uniform3d_1m"]
        P2 = torch.from_numpy(gen_points(w2, seed_offset=rank)).to(f"cuda:{local}")
        tri.triangulate(P2, k=w2["k"], sample_frac=w2["frac"], fetch=False)
        sec_ms, _ = steps_ms(P2, w2["k"], max(args.steps // 4, 3))
        st2 = tri.stats().as_dict()
        pl2_ms, _ = steps_ms(P2, 1, max(args.steps // 4, 3))
        secondary = {"workload": "uniform3d_1m", "n": w2["n"], "k": w2["k"], "sample_frac": w2["frac"],
                     "value": job_value(w2["n"], world, max_over_ranks(sum(sec_ms) / len(sec_ms), dist,
                                                                        f"cuda:{local}")),
                     "ms_per_step": sum(sec_ms) / len(sec_ms),
                     "plain_path": job_value(w2["n"], world, max_over_ranks(sum(pl2_ms) / len(pl2_ms), dist,
                                                                            f"cuda:{local}")),
                     **{k: st2[k] for k in ("border_vertices", "imbalance", "cv", "o_dt")}}
        del P2

    # ---------------- latency under load: a short serving leg on this GPU
    latency = None
    if not args.no_serve_leg and rank == 0 and w["dim"] == 3:
        tri.close()
        torch.cuda.synchronize()
        spts = serving_jobs(args.serve_jobs, seed=5)
        latency = serving_leg(local, spts, plain_service_times(local, spts), load=0.8, seed=5)
        tri = None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # ---------------- roofline of the dominant kernel (live CUDA-event times)
    peaks, peak_src = load_peaks()
    fma = {"fp32": fma_rate(local, 32, 5), "fp64": fma_rate(local, 64, 5)}
    roofline = make_roofline(prof_tot, prof_step_ms, units, w["dim"], nprof, peaks, peak_src, fma, n=n)
    kernels = {k: {"ms_per_step": round(v["ms"] / nprof, 3), "launches_per_step": v["launches"] / nprof}
               for k, v in prof_tot.items()}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(w)

    line = {
        "metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "dim": w["dim"], "k": w["k"], "sample_frac": sample_frac,
                   "divide": args.divide + (" recursive bisection" if args.recursive else ""),
                   "primitive": "grid", "weight": args.weight or "log", "neighbors": True,
                   "partitioner": "multilevel" if args.partitioner == "ml" else "label propagation",
                   "rounds": "host-driven (profile mode)" if args.host_rounds else "one CUDA graph per engine run",
                   "l2": "flushed before every step (256 MiB write); working set > L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "e2e": e2e, "plain_path": plain, "divide_comparator": comparator, "partitioner_comparator": part_cmp,
        "latency": latency,
        "secondary": secondary, "roofline": roofline, "fma_peaks_tflops": fma, "cpu_baseline": cpu,
        "clocks": clocks, "gpu_launches": int(launches),
        "stats": {k: stats[k] for k in ("simplices", "eta", "border_vertices", "border_simplices", "imbalance",
                                         "cv", "o_dt", "cut_weight", "rounds_max", "exact_calls", "ms_phase")},
        "triangulated_points_per_step": units,
        "kernels": kernels, "wall_s": wall,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def parse_frac(arg, default, n: int):
    """Sample size of Sec. 4.2 as the library's sample_frac: a fraction of n,
    'sqrt' (eta = ceil(sqrt n), the paper's default; the library reads 0 so)
    or 'logn' (eta = ceil(log2 n), passed as a fraction that rounds up to it)."""
    if arg is None:
        return default
    if arg == "sqrt":
        return 0.0
    if arg == "logn":
        return (math.ceil(math.log2(n)) - 0.5) / n
    return float(arg)


def serving_jobs(jobs: int, seed: int = 5):
    """The serving workload: `jobs` 3D jobs, sizes log-uniform in
    1,000..2,000,000 points, half uniform, half clustered."""
    sizes, kinds, seeds = pointsets.serve_jobs(jobs, seed=seed)
    return [pointsets.job_points(sizes[i], kinds[i], seeds[i]) for i in range(jobs)]


def plain_service_times(device: int, pts) -> list:
    """The plain path (one context, k = 1, no batching) on every job back to
    back, simplices copied to the host: seconds per job."""
    from paper_1902_07554_gb300 import Triangulator
    with Triangulator(device) as plain:
        plain.triangulate(pts[0][:5000], k=1, fetch=False)
        service = []
        for P in pts:
            t = time.perf_counter()
            plain.triangulate(P, k=1, fetch=True)
            service.append(time.perf_counter() - t)
    return service


def serving_leg(device: int, pts, service, load: float, seed: int = 5, budget: float = 120e9) -> dict:
    """Latency under load on this GPU: the jobs arrive as a Poisson stream at
    `load` x the plain path's measured capacity.  Served form: the
    continuous-batching server (one resident engine, jobs admitted at round
    boundaries, device memory from `budget`).  Plain path: one context, k = 1,
    no batching, jobs taken first in, first out under the SAME arrival times
    (replayed on the clock, not simulated).  Latency = arrival to simplices
    on the host."""
    from paper_1902_07554_gb300 import Triangulator
    from paper_1902_07554_gb300.serve import Job, Server, poisson_arrivals
    jobs = len(pts)
    total = int(sum(len(p) for p in pts))
    cap = total / sum(service)
    rate = load * cap / (total / jobs)
    arr = poisson_arrivals(jobs, rate, seed)
    lat = []
    with Triangulator(device) as plain:
        plain.triangulate(pts[0][:5000], k=1, fetch=False)
        t0 = time.perf_counter()
        for a, P in zip(arr, pts):
            delay = a - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            plain.triangulate(P, k=1, fetch=True)
            lat.append(time.perf_counter() - t0 - a)
        span = time.perf_counter() - t0 - arr[0]
    lat = np.array(lat)
    plain_sum = {"throughput_mpts": total / span / 1e6, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                 "p99_ms": float(np.percentile(lat, 99) * 1e3), "capacity_mpts": cap / 1e6}
    srv = Server(device=device, dim=3, budget_bytes=budget, keep_results=False)
    served = srv.run([Job(float(arr[i]), i, pts[i]) for i in range(jobs)])
    keep = ("throughput_mpts", "p50_ms", "p99_ms", "mean_ms", "makespan_s", "failed", "capacity_points",
            "peak_running_points", "device_gb", "quanta", "rounds", "launches", "model_bytes_per_point")
    return {"jobs": jobs, "points": total, "offered_load": load, "budget_gb": budget / 1e9,
            "served": {k: served[k] for k in keep if k in served}, "plain": plain_sum}


if __name__ == "__main__":
    sys.exit(main())
