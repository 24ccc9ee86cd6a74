"""Seeded synthetic point sets shaped like the paper's workloads.

This module only draws random numbers.  It holds none of the triangulation
arithmetic, so both the CPU oracle and the CUDA path can take their inputs
from it without sharing any of the method's code.

The paper evaluates on uniform points in the unit cube, normally distributed
points, random "bubbles" (Gaussian blobs) and an ellipsoid surface (Sec. 4,
Table 2).  Its real data set (Gaia DR2) is not available; the clustered
generator below (blobs plus a noisy 2.5D surface) stands in for the
structured inputs.  All arrays are float64, row-major (n, dim), and point i
keeps global index i.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "uniform",
    "normal",
    "clustered",
    "grid",
    "cocircular",
    "batch_instances",
    "serve_jobs",
    "WORKLOADS",
    "workload",
]


def uniform(n: int, dim: int, seed: int) -> np.ndarray:
    """n points uniform in [0,1]^dim."""
    rng = np.random.default_rng(seed)
    return rng.random((n, dim), dtype=np.float64)


def normal(n: int, dim: int, seed: int, mu: float = 0.5, sigma: float = 0.1) -> np.ndarray:
    """n points N(mu, sigma^2) per coordinate, unclipped."""
    rng = np.random.default_rng(seed)
    return rng.normal(mu, sigma, size=(n, dim)).astype(np.float64)


def clustered(n: int, seed: int, nblobs: int = 50, surface_frac: float = 0.2,
              sigma_lo: float = 0.01, sigma_hi: float = 0.05) -> np.ndarray:
    """3D clustered points: Gaussian blobs plus a noisy heightfield surface.

    (1 - surface_frac) of the points come from `nblobs` isotropic Gaussian
    blobs with centres uniform in [0,1]^3 and sigma uniform in
    [sigma_lo, sigma_hi]; each point picks a blob uniformly and is re-drawn
    until it falls inside [0,1]^3.  The rest lie on
    z = 0.5 + sum_j a_j sin(2 pi (fx_j x + fy_j y) + phi_j) + N(0, 1e-3)
    over (x, y) uniform in [0,1]^2, with 8 terms, a_j ~ U[0, 0.05],
    f ~ U{1..4}, phi ~ U[0, 2 pi).  The rows are shuffled.
    """
    rng = np.random.default_rng(seed)
    n_surf = int(round(n * surface_frac))
    n_blob = n - n_surf
    centres = rng.random((nblobs, 3))
    sig = rng.uniform(sigma_lo, sigma_hi, size=nblobs)
    out = np.empty((n, 3), dtype=np.float64)
    filled = 0
    while filled < n_blob:
        m = (n_blob - filled) + 64
        b = rng.integers(0, nblobs, size=m)
        p = centres[b] + rng.standard_normal((m, 3)) * sig[b, None]
        ok = np.all((p >= 0.0) & (p <= 1.0), axis=1)
        p = p[ok][: n_blob - filled]
        out[filled:filled + len(p)] = p
        filled += len(p)
    if n_surf:
        amp = rng.uniform(0.0, 0.05, size=8)
        fx = rng.integers(1, 5, size=8)
        fy = rng.integers(1, 5, size=8)
        ph = rng.uniform(0.0, 2.0 * math.pi, size=8)
        xy = rng.random((n_surf, 2))
        z = np.full(n_surf, 0.5)
        for j in range(8):
            z += amp[j] * np.sin(2.0 * math.pi * (fx[j] * xy[:, 0] + fy[j] * xy[:, 1]) + ph[j])
        z += rng.normal(0.0, 1e-3, size=n_surf)
        out[n_blob:, 0:2] = xy
        out[n_blob:, 2] = z
    perm = rng.permutation(n)
    return np.ascontiguousarray(out[perm])


def grid(shape, seed: int | None = None, jitter: float = 0.0) -> np.ndarray:
    """Integer lattice points (a maximally degenerate input: many cocircular /
    cospherical and collinear subsets).  Optionally shuffled by `seed`."""
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    pts = np.stack([m.ravel() for m in mesh], axis=1)
    if jitter:
        rng = np.random.default_rng(seed)
        pts = pts + rng.uniform(-jitter, jitter, size=pts.shape)
    if seed is not None:
        rng = np.random.default_rng(seed)
        pts = pts[rng.permutation(len(pts))]
    return np.ascontiguousarray(pts)


def cocircular(n: int, seed: int) -> np.ndarray:
    """n distinct integer points exactly on the circle x^2 + y^2 = 5^4 = 625
    (plus scaled copies are exact in float64).  Used for degenerate tests."""
    pts = []
    r2 = 625
    for x in range(-25, 26):
        for y in range(-25, 26):
            if x * x + y * y == r2:
                pts.append((float(x), float(y)))
    pts = np.array(pts, dtype=np.float64)
    rng = np.random.default_rng(seed)
    pts = pts[rng.permutation(len(pts))]
    return np.ascontiguousarray(pts[: min(n, len(pts))])


def batch_instances(count: int = 4096, seed: int = 4, lo: int = 256, hi: int = 65536,
                    dim: int = 2):
    """Many independent 2D instances with log-uniform sizes in [lo, hi].

    Instance i draws its size from the batch seed and then, from seed+i,
    whether it is uniform in [0,1]^2 or N(0.5, 0.1^2) (unclipped).
    Returns (points (N,dim), offsets (count+1,), kinds list).
    """
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    offsets = np.zeros(count + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    pts = np.empty((int(offsets[-1]), dim), dtype=np.float64)
    kinds = []
    for i in range(count):
        r = np.random.default_rng(seed + 1 + i)
        kind = "uniform" if r.random() < 0.5 else "normal"
        kinds.append(kind)
        m = int(sizes[i])
        if kind == "uniform":
            pts[offsets[i]:offsets[i + 1]] = r.random((m, dim))
        else:
            pts[offsets[i]:offsets[i + 1]] = r.normal(0.5, 0.1, size=(m, dim))
    return pts, offsets, kinds


def batch_instance(i: int, count: int = 4096, seed: int = 4, lo: int = 256, hi: int = 65536,
                   dim: int = 2) -> np.ndarray:
    """Instance i of batch_instances(count, seed, lo, hi, dim) alone (the same
    points, without generating the others)."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    m = int(np.clip(sizes, lo, hi)[i])
    r = np.random.default_rng(seed + 1 + i)
    if r.random() < 0.5:
        return r.random((m, dim))
    return r.normal(0.5, 0.1, size=(m, dim))


def serve_jobs(count: int, seed: int = 5, lo: int = 1000, hi: int = 2_000_000):
    """Job sizes log-uniform in [lo, hi] and a kind per job (uniform or
    clustered).  Arrival times are drawn by the serving driver from the offered
    load, so this returns only (sizes, kinds, per-job seeds)."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    kinds = np.where(rng.random(count) < 0.5, "uniform", "clustered")
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return sizes, list(kinds), seeds


def job_points(size: int, kind: str, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform(int(size), 3, int(seed))
    return clustered(int(size), int(seed))


# Named workloads (the paper's configurations restated with sizes).
WORKLOADS = {
    "uniform2d_10k": dict(dim=2, n=10_000, kind="uniform", seed=1, k=4, frac=0.01),
    "uniform3d_1m": dict(dim=3, n=1_000_000, kind="uniform", seed=2, k=16, frac=0.005),
    "clustered3d_4m": dict(dim=3, n=4_000_000, kind="clustered", seed=3, k=64, frac=0.005),
}


def workload(name: str, n: int | None = None) -> np.ndarray:
    w = WORKLOADS[name]
    m = w["n"] if n is None else n
    if w["kind"] == "uniform":
        return uniform(m, w["dim"], w["seed"])
    if w["kind"] == "normal":
        return normal(m, w["dim"], w["seed"])
    return clustered(m, w["seed"])
