"""CPU oracle for the sample-based divide-and-conquer Delaunay triangulation.

TEST INFRASTRUCTURE ONLY.  This package is imported by the tests, by the
package smoke check and by the benchmark's CPU-baseline leg; the product path
never imports it, and it imports nothing from the product package.

Contents
--------
* ``delaunay``   -- DT(P) under the symbolic perturbation (Sec. 2.1), by
  incremental Bowyer-Watson in plain C (``dt_oracle.c``).  Because the
  divide-and-conquer method is exact (Alg. 1), its final output must equal
  this set for every k, sample and seed.
* ``bruteforce`` -- every (d+1)-subset with an empty perturbed circumsphere
  (tiny inputs only): the definition itself.
* ``predicates`` -- orient / insphere / closer signs on index tuples.
* ``nearest``    -- exact nearest sample site (Alg. 2, assignment loop).
* ``neighbors``  -- the neighbour relation of a set of simplices (the state
  the merge's neighbourhood update must reach).
* the divide-step references in ``oracle.divide`` (sampling, graph, weights,
  partition invariants, labels, kd median split, border set, merge rule and
  the partition-quality metrics of Sec. 4.6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dt_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.RLock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags; no -march)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-g", "-fPIC", "-shared", "-frounding-math",
           "-ffp-contract=off", "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, i32, p = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            L.or_dt_build.restype = i64
            L.or_dt_build.argtypes = [i32, i64, p, p]
            L.or_dt_fetch.restype = i64
            L.or_dt_fetch.argtypes = [p, i64, p]
            L.or_dt_fetch_mesh.restype = i64
            L.or_dt_fetch_mesh.argtypes = [p, p]
            L.or_predicates.restype = i32
            L.or_predicates.argtypes = [i32, i64, p, p, i32, i64, p, p]
            L.or_dt_bruteforce.restype = i64
            L.or_dt_bruteforce.argtypes = [i32, i64, p, p, p, i64]
            L.or_nearest.restype = i32
            L.or_nearest.argtypes = [i32, i64, p, i64, p, p, p]
            L.or_exact_calls.restype = ctypes.c_long
            L.or_interval_selftest.restype = i32
            _lib = L
        return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


class OracleError(RuntimeError):
    pass


_ERR = {-1: "degenerate input (no d+1 affinely independent points)",
        -2: "duplicate point"}


def delaunay(points: np.ndarray, gid: np.ndarray | None = None, mesh: bool = False):
    """DT(points) as an (m, d+1) int64 array of global indices (each row
    sorted ascending, rows sorted lexicographically).  `gid` gives the global
    index of each row of `points` (used both as the perturbation rank and for
    the output); default: 0..n-1.  With mesh=True also returns the raw mesh
    (vertices with -1 for the infinite vertex, neighbour links, local ids)."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    n, D = P.shape
    g = None if gid is None else np.ascontiguousarray(gid, dtype=np.int64)
    L = lib()
    with _lock:
        cnt = L.or_dt_build(D, n, _ptr(P), _ptr(g))
        if cnt < 0:
            raise OracleError(_ERR.get(int(cnt), f"internal error {cnt}"))
        out = np.empty((cnt, D + 1), dtype=np.int64)
        k = L.or_dt_fetch(_ptr(out), cnt, _ptr(g))
        assert k == cnt
        if not mesh:
            return out
        ns = L.or_dt_fetch_mesh(None, None)
        v = np.empty((ns, D + 1), dtype=np.int32)
        nb = np.empty((ns, D + 1), dtype=np.int32)
        L.or_dt_fetch_mesh(_ptr(v), _ptr(nb))
        return out, v, nb


def bruteforce(points: np.ndarray, gid: np.ndarray | None = None) -> np.ndarray:
    """The definition: all (d+1)-subsets with nonzero orientation and an
    empty perturbed circumsphere.  O(n^(d+2)); tiny inputs only.  Returns
    local indices mapped through gid like ``delaunay``."""
    P = np.ascontiguousarray(points, dtype=np.float64)
    n, D = P.shape
    g = None if gid is None else np.ascontiguousarray(gid, dtype=np.int64)
    cap = 4 * n * n + 64
    out = np.empty((cap, D + 1), dtype=np.int64)
    with _lock:
        k = lib().or_dt_bruteforce(D, n, _ptr(P), _ptr(g), _ptr(out), cap)
    if k < 0:
        raise OracleError("brute force capacity exceeded")
    out = out[:k]
    if g is not None:
        out = np.sort(g[out], axis=1)
        out = out[np.lexsort(out.T[::-1])]
    return out


def predicates(points: np.ndarray, kind: str, tuples: np.ndarray,
               gid: np.ndarray | None = None) -> np.ndarray:
    """Exact predicate signs on index tuples.

    kind 'orient'  : tuples (m, d+1) -> sign of det[p_i - p_0]
    kind 'insphere': tuples (m, d+2) -> perturbed insphere of point d+1
                     against simplex 0..d (orientation normalised first;
                     0 only when the simplex is flat)
    kind 'insphere_raw': unperturbed sign of (-1)^d det[p_i - q, |p_i - q|^2]
    kind 'closer'  : tuples (m, 3) (p, a, b) -> sign(|p-a|^2 - |p-b|^2)
    """
    P = np.ascontiguousarray(points, dtype=np.float64)
    n, D = P.shape
    code = {"orient": 0, "insphere": 1, "insphere_raw": 2, "closer": 3}[kind]
    T = np.ascontiguousarray(tuples, dtype=np.int32)
    out = np.empty(len(T), dtype=np.int8)
    g = None if gid is None else np.ascontiguousarray(gid, dtype=np.int64)
    with _lock:
        lib().or_predicates(D, n, _ptr(P), _ptr(g), code, len(T), _ptr(T), _ptr(out))
    return out


def nearest(queries: np.ndarray, sites: np.ndarray, site_rank: np.ndarray | None = None) -> np.ndarray:
    """Index of the exactly nearest site for every query (ties: smaller rank)."""
    Q = np.ascontiguousarray(queries, dtype=np.float64)
    S = np.ascontiguousarray(sites, dtype=np.float64)
    D = Q.shape[1]
    r = np.arange(len(S), dtype=np.int64) if site_rank is None else np.ascontiguousarray(site_rank, dtype=np.int64)
    out = np.empty(len(Q), dtype=np.int32)
    with _lock:
        lib().or_nearest(D, len(Q), _ptr(Q), len(S), _ptr(S), _ptr(r), _ptr(out))
    return out


def exact_calls() -> int:
    return int(lib().or_exact_calls())


def interval_selftest() -> bool:
    return bool(lib().or_interval_selftest())


# ---------------------------------------------------------------------------
# Invariants of a triangulation given as sorted vertex tuples (Sec. 2.1).
# ---------------------------------------------------------------------------
def faces(simplices: np.ndarray) -> np.ndarray:
    """All (d)-vertex facets of the simplices, with multiplicity, each row sorted."""
    S = np.asarray(simplices)
    D1 = S.shape[1]
    parts = [np.delete(S, i, axis=1) for i in range(D1)]
    return np.sort(np.concatenate(parts, axis=0), axis=1)


def unique_rows(a: np.ndarray):
    a = np.ascontiguousarray(a)
    if len(a) == 0:
        return a, np.zeros(0, dtype=np.int64)
    u, cnt = np.unique(a, axis=0, return_counts=True)
    return u, cnt


def edges(simplices: np.ndarray) -> np.ndarray:
    S = np.asarray(simplices)
    D1 = S.shape[1]
    pairs = [S[:, [i, j]] for i in range(D1) for j in range(i + 1, D1)]
    e = np.sort(np.concatenate(pairs, axis=0), axis=1)
    return np.unique(e, axis=0)


def neighbors(simplices: np.ndarray) -> np.ndarray:
    """The neighbour relation of a triangulation, by its definition (the
    neighbourhood update of Alg. 1 must end with it): entry [r, j] is the
    row sharing every vertex of row r except row r's j-th, -1 when no other
    row has that facet (a hull facet).  Raises if a facet is in more than
    two rows."""
    S = np.asarray(simplices, dtype=np.int64)
    m, D1 = S.shape if S.ndim == 2 else (0, 1)
    out = -np.ones((m, D1), dtype=np.int64)
    if m == 0:
        return out
    F = np.concatenate([np.sort(np.delete(S, j, axis=1), axis=1) for j in range(D1)])
    slot = np.concatenate([np.arange(m) * D1 + j for j in range(D1)])
    order = np.lexsort(F.T[::-1])
    F, slot = F[order], slot[order]
    same = np.all(F[1:] == F[:-1], axis=1)
    if len(same) > 1:
        assert not np.any(same[1:] & same[:-1]), "a facet lies in more than two simplices"
    i = np.nonzero(same)[0]
    a, b = slot[i], slot[i + 1]
    flat = out.reshape(-1)
    flat[a] = b // D1
    flat[b] = a // D1
    return out


def hull_vertex_count(simplices: np.ndarray) -> int:
    """Number of vertices on hull facets (facets used by exactly one simplex)."""
    f, cnt = unique_rows(faces(simplices))
    return int(len(np.unique(f[cnt == 1])))


def check_combinatorics(simplices: np.ndarray, n: int) -> dict:
    """Euler-type identities every triangulation of n points must satisfy.

    2D: T = 2n - 2 - h and E = 3n - 3 - h.
    3D: V - E + F - T = 1, hull facets = 2h - 4.
    Every facet is used once (hull) or twice (interior); every point is a vertex.
    Returns the counts; raises AssertionError on violation."""
    S = np.asarray(simplices)
    D = S.shape[1] - 1
    assert len(np.unique(S)) == n, "not every point is a vertex"
    f, cnt = unique_rows(faces(S))
    assert cnt.max() <= 2, "a facet is shared by more than two simplices"
    h = int(len(np.unique(f[cnt == 1])))
    T = len(S)
    E = len(edges(S))
    if D == 2:
        assert T == 2 * n - 2 - h, (T, n, h)
        assert E == 3 * n - 3 - h, (E, n, h)
        return dict(T=T, E=E, h=h)
    F = len(f)
    hull_f = int((cnt == 1).sum())
    assert n - E + F - T == 1, (n, E, F, T)
    assert hull_f == 2 * h - 4, (hull_f, h)
    return dict(T=T, E=E, F=F, h=h, hull_facets=hull_f)


def check_volume(points: np.ndarray, simplices: np.ndarray, hull_volume: float, rtol=1e-9) -> float:
    """Sum of |simplex volume| equals the hull volume (floating point)."""
    P = np.asarray(points, dtype=np.float64)
    S = np.asarray(simplices)
    D = S.shape[1] - 1
    base = P[S[:, 0]]
    M = np.stack([P[S[:, i]] - base for i in range(1, D + 1)], axis=1)
    vol = np.abs(np.linalg.det(M)).sum() / (2.0 if D == 2 else 6.0)
    assert abs(vol - hull_volume) <= rtol * max(1.0, abs(hull_volume)), (vol, hull_volume)
    return float(vol)


def check_locally_delaunay(points: np.ndarray, simplices: np.ndarray,
                           gid: np.ndarray | None = None) -> int:
    """Every interior facet is locally Delaunay: the vertex of one neighbour
    opposite the shared facet is not inside the other's perturbed
    circumsphere.  Returns the number of interior facets checked."""
    S = np.asarray(simplices, dtype=np.int64)
    D1 = S.shape[1]
    m = len(S)
    fs, owner, opp = [], [], []
    for i in range(D1):
        fs.append(np.sort(np.delete(S, i, axis=1), axis=1))
        owner.append(np.arange(m))
        opp.append(S[:, i])
    F = np.concatenate(fs)
    own = np.concatenate(owner)
    op = np.concatenate(opp)
    order = np.lexsort(F.T[::-1])
    F, own, op = F[order], own[order], op[order]
    same = np.all(F[1:] == F[:-1], axis=1)
    idx = np.nonzero(same)[0]
    if len(idx) == 0:
        return 0
    a_owner = own[idx]
    b_opp = op[idx + 1]
    b_owner = own[idx + 1]
    a_opp = op[idx]
    t1 = np.concatenate([S[a_owner], b_opp[:, None]], axis=1)
    t2 = np.concatenate([S[b_owner], a_opp[:, None]], axis=1)
    r1 = predicates(points, "insphere", t1, gid)
    r2 = predicates(points, "insphere", t2, gid)
    assert np.all(r1 < 0) and np.all(r2 < 0), "non-Delaunay interior facet"
    return int(len(idx))
