"""Schedule autotuning of the insertion engine for a workload shape.

The engine's schedule has five knobs in dt_config: brio_growth (batch growth
x 100), brio_drain (how far the active set drains before the next batch),
first_batch (points per instance in the first batch), nominate_rings (the
neighbour rings in which a nominee must hold the strongest pick: the queue of
regions grown per round) and cavity_blocks (the tile of the region-growth and
insertion kernels: thread blocks per SM).  The best
setting depends on the shape of the work -- one large instance, a few
partitions, or thousands of small batched instances -- so `autotune` times a
small grid of candidates on a representative input through the library's
own calls, applies the fastest to the context, and remembers it per shape.

Everything runs through the C ABI; Python only times and chooses.
"""
from __future__ import annotations

import itertools
import math
import time

import numpy as np

# round schedule (BRIO growth, drain, first batch), nominee queue policy (the
# rings a nominee must hold the strongest pick in) and the cavity tiles (thread
# blocks per SM of the region-growth and insertion kernels)
DEFAULT_GRID = {"brio_growth": (125, 150, 200), "brio_drain": (4, 8), "first_batch": (32, 128),
                "nominate_rings": (1, 2), "cavity_blocks": (8, 16)}

_cache: dict = {}


def shape_key(points, offsets=None, k: int = 1) -> tuple:
    """The shape a schedule is tuned for: dimension, instance count and the
    mean instance size, both rounded to powers of two, and k."""
    P = np.asarray(points) if not hasattr(points, "shape") else points
    n, dim = int(P.shape[0]), int(P.shape[1])
    count = 1 if offsets is None else len(offsets) - 1
    mean = n / max(count, 1)
    return (dim, int(round(math.log2(max(count, 1)))), int(round(math.log2(max(mean, 1.0)))), int(k))


def candidates(grid: dict | None = None) -> list[dict]:
    g = DEFAULT_GRID if grid is None else grid
    names = sorted(g)
    return [dict(zip(names, vals)) for vals in itertools.product(*(g[nm] for nm in names))]


def autotune(tri, points, offsets=None, k: int = 1, sample_frac: float = 0.0, grid: dict | None = None,
             reps: int = 2, use_cache: bool = True, clock=time.perf_counter) -> dict:
    """Times every candidate schedule on `points` (a batch when `offsets` is
    given), `reps` runs each after one untimed run, applies the fastest to
    `tri` and returns {"best": config, "ms": best time, "table": [(config,
    ms), ...]}.  Ties go to the earlier candidate.  With use_cache, a shape
    tuned before is applied without timing."""
    key = shape_key(points, offsets, k)
    if use_cache and key in _cache:
        best = _cache[key]
        tri.configure(**best["best"])
        return dict(best, cached=True)

    def run():
        if offsets is None:
            tri.triangulate(points, k=k, sample_frac=sample_frac, fetch=False)
        else:
            tri.triangulate_batch(points, offsets, fetch=False)

    table = []
    for cand in candidates(grid):
        tri.configure(**cand)
        run()
        ts = []
        for _ in range(max(1, reps)):
            t = clock()
            run()
            ts.append(clock() - t)
        table.append((cand, 1e3 * min(ts)))
    best_cfg, best_ms = min(table, key=lambda e: e[1])   # min keeps the first of equal times
    tri.configure(**best_cfg)
    out = {"best": best_cfg, "ms": best_ms, "table": table, "key": key}
    if use_cache:
        _cache[key] = out
    return dict(out, cached=False)


def clear_cache():
    _cache.clear()
