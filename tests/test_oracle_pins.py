"""Pins for the CPU oracle against things other than itself.

* predicate signs vs. exact rational determinants written out in Python
  (``fractions.Fraction``) -- the textbook definitions, independent of the C
  big-integer code;
* the symbolic perturbation vs. an explicit perturbation of the lifting map
  with concrete infinitesimals (powers of 2^-80) evaluated exactly;
* incremental Bowyer-Watson vs. brute force (the definition of DT(P),
  Sec. 2.1), vs. a pure-Python brute force, and vs. scipy/qhull on random
  inputs in general position;
* Euler / hull identities and the volume identity on larger outputs;
* a hand-derived golden case (tests/golden/square_sos.txt).
"""
import itertools
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import pointsets

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def det(M):
    n = len(M)
    if n == 1:
        return M[0][0]
    s = Fr(0)
    for j in range(n):
        minor = [row[:j] + row[j + 1:] for row in M[1:]]
        s += (-1) ** j * M[0][j] * det(minor)
    return s


def fr_orient(pts):
    p0 = [Fr(x) for x in pts[0]]
    M = [[Fr(x) - p0[c] for c, x in enumerate(p)] for p in pts[1:]]
    return (det(M) > 0) - (det(M) < 0)


def fr_insphere_raw(pts, q, lift_extra=None):
    D = len(q)
    qf = [Fr(x) for x in q]
    M = []
    for i, p in enumerate(pts):
        d = [Fr(x) - qf[c] for c, x in enumerate(p)]
        lift = sum(x * x for x in d)
        if lift_extra is not None:
            lift += lift_extra[i]
        M.append(d + [lift])
    v = det(M) * (-1) ** D
    return (v > 0) - (v < 0)


def fr_insphere_perturbed(pts, q, gids, gq):
    """(-1)^D det[p_i - q, |p_i - q|^2 + delta_i - delta_q] with
    delta = eps^(2^j), j = position by descending global index, eps = 2^-80."""
    order = sorted(list(gids) + [gq], reverse=True)
    eps = Fr(1, 2 ** 80)
    delta = {g: eps ** (2 ** j) for j, g in enumerate(order)}
    extra = [delta[g] - delta[gq] for g in gids]
    return fr_insphere_raw(pts, q, extra)


def positively_oriented(pts, idx):
    o = fr_orient([pts[i] for i in idx])
    if o < 0:
        idx = [idx[1], idx[0]] + list(idx[2:])
    return idx, o


def py_bruteforce(P, gid):
    n, D = P.shape
    out = []
    for comb in itertools.combinations(range(n), D + 1):
        idx, o = positively_oriented(P, list(comb))
        if o == 0:
            continue
        ok = True
        for q in range(n):
            if q in comb:
                continue
            if fr_insphere_perturbed([P[i] for i in idx], P[q], [gid[i] for i in idx], gid[q]) > 0:
                ok = False
                break
        if ok:
            out.append(sorted(gid[i] for i in comb))
    out.sort()
    return np.array(out, dtype=np.int64).reshape(-1, D + 1)


# ---------------------------------------------------------------- tests
def test_interval_rounding_selftest(orc):
    assert orc.interval_selftest()


@pytest.mark.parametrize("D", [2, 3])
def test_orient_and_insphere_match_rationals_random(orc, D):
    rng = np.random.default_rng(11 + D)
    P = rng.random((60, D))
    tup_o = np.array([rng.choice(60, D + 1, replace=False) for _ in range(300)], dtype=np.int32)
    tup_i = np.array([rng.choice(60, D + 2, replace=False) for _ in range(300)], dtype=np.int32)
    so = orc.predicates(P, "orient", tup_o)
    si = orc.predicates(P, "insphere_raw", tup_i)
    for t, s in zip(tup_o, so):
        assert s == fr_orient([P[i] for i in t])
    for t, s in zip(tup_i, si):
        assert s == fr_insphere_raw([P[i] for i in t[:-1]], P[t[-1]])


@pytest.mark.parametrize("D", [2, 3])
def test_predicates_near_and_exactly_degenerate(orc, D):
    """Cocircular / cospherical and coplanar tuples (exact zeros), then the
    same tuples with one coordinate moved by one ulp (tiny nonzero values the
    floating-point filter cannot decide)."""
    base = pointsets.grid((3,) * D).astype(np.float64) * 0.1 + 0.3   # non-integers
    rng = np.random.default_rng(5)
    before = orc.exact_calls()
    for trial in range(120):
        P = base.copy()
        if trial % 2:
            i, c = rng.integers(len(P)), rng.integers(D)
            P[i, c] = np.nextafter(P[i, c], np.inf if rng.random() < 0.5 else -np.inf)
        ti = rng.choice(len(P), D + 2, replace=False).astype(np.int32)
        to = ti[: D + 1]
        assert orc.predicates(P, "orient", to[None])[0] == fr_orient([P[i] for i in to])
        assert orc.predicates(P, "insphere_raw", ti[None])[0] == fr_insphere_raw([P[i] for i in ti[:-1]], P[ti[-1]])
    assert orc.exact_calls() > before, "the exact fallback was never exercised"


def test_predicates_wide_exponent_range(orc):
    """Coordinates spanning hundreds of binary orders of magnitude."""
    P = np.array([[1e-200, 0.0], [1.0, 1e-150], [0.0, 1.0], [1.0, 1.0], [1e100, 1e-100]])
    for t in itertools.permutations(range(5), 4):
        t = np.array(t, dtype=np.int32)
        assert orc.predicates(P, "insphere_raw", t[None])[0] == fr_insphere_raw([P[i] for i in t[:-1]], P[t[-1]])
        assert orc.predicates(P, "orient", t[None, :3])[0] == fr_orient([P[i] for i in t[:3]])


@pytest.mark.parametrize("D", [2, 3])
def test_perturbation_matches_explicit_infinitesimals(orc, D):
    """Integer-grid tuples (mostly exactly cospherical) with shuffled global
    indices: the oracle's perturbed insphere equals the sign of the lifted
    determinant with concrete infinitesimal lifts added."""
    P = pointsets.grid((3,) * D)
    rng = np.random.default_rng(21 + D)
    gid = rng.permutation(len(P)).astype(np.int64) * 7 + 3
    checked = 0
    while checked < 150:
        t = rng.choice(len(P), D + 2, replace=False)
        s = list(t[: D + 1])
        idx, o = positively_oriented(P, s)
        if o == 0:
            continue
        tup = np.array(idx + [t[-1]], dtype=np.int32)
        got = orc.predicates(P, "insphere", tup[None], gid)[0]
        want = fr_insphere_perturbed([P[i] for i in idx], P[t[-1]], [gid[i] for i in idx], gid[t[-1]])
        assert got == want, (tup, got, want)
        checked += 1


def test_closer_matches_rationals(orc):
    rng = np.random.default_rng(3)
    P = np.round(rng.random((40, 3)) * 8) / 8    # many exact ties
    tup = np.array([rng.choice(40, 3, replace=False) for _ in range(400)], dtype=np.int32)
    got = orc.predicates(P, "closer", tup)
    for t, g in zip(tup, got):
        p, a, b = (P[i] for i in t)
        v = sum((Fr(p[c]) - Fr(a[c])) ** 2 for c in range(3)) - sum((Fr(p[c]) - Fr(b[c])) ** 2 for c in range(3))
        assert g == (v > 0) - (v < 0)


@pytest.mark.parametrize("D,n,shape", [(2, 9, (3, 3)), (2, 10, None), (3, 8, (2, 2, 2)), (3, 9, None)])
def test_bruteforce_matches_pure_python(orc, D, n, shape):
    if shape is not None:
        P = pointsets.grid(shape, seed=2)
    else:
        P = pointsets.uniform(n, D, 4)
    gid = np.random.default_rng(9).permutation(len(P)).astype(np.int64)
    want = py_bruteforce(P, gid)
    assert np.array_equal(orc.bruteforce(P, gid), want)
    assert np.array_equal(orc.delaunay(P, gid), want)


def test_golden_square(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "square_sos.txt")) if l.strip() and not l.startswith("#")]
    P = np.array([[float(x) for x in r] for r in rows[:4]])
    want = np.array([[int(x) for x in r] for r in rows[4:]], dtype=np.int64)
    assert np.array_equal(orc.delaunay(P), want)
    assert np.array_equal(orc.bruteforce(P), want)


@pytest.mark.parametrize("D,n", [(2, 40), (3, 14)])
@pytest.mark.parametrize("seed", range(4))
def test_bowyer_watson_matches_bruteforce_random(orc, D, n, seed):
    P = pointsets.uniform(n, D, 100 + seed)
    gid = np.random.default_rng(seed).permutation(n).astype(np.int64)
    assert np.array_equal(orc.delaunay(P, gid), orc.bruteforce(P, gid))


@pytest.mark.parametrize("shape", [(6, 5), (7, 3), (3, 3, 3), (4, 3, 2), (2, 2, 5)])
def test_bowyer_watson_matches_bruteforce_degenerate(orc, shape):
    for seed in range(3):
        P = pointsets.grid(shape, seed=seed)
        gid = np.random.default_rng(seed).permutation(len(P)).astype(np.int64)
        a = orc.delaunay(P, gid)
        assert np.array_equal(a, orc.bruteforce(P, gid))
        orc.check_combinatorics(a, len(P))


def test_bowyer_watson_cocircular(orc):
    P = pointsets.cocircular(20, 1)
    for seed in range(3):
        gid = np.random.default_rng(seed).permutation(len(P)).astype(np.int64)
        a = orc.delaunay(P, gid)
        assert np.array_equal(a, orc.bruteforce(P, gid))
        assert len(a) == len(P) - 2           # a convex polygon: n - 2 triangles


@pytest.mark.parametrize("D,n", [(2, 3000), (3, 800)])
def test_bowyer_watson_matches_qhull(orc, D, n):
    spatial = pytest.importorskip("scipy.spatial")
    for seed in range(2):
        P = pointsets.uniform(n, D, 200 + seed)
        s = np.sort(spatial.Delaunay(P).simplices, axis=1).astype(np.int64)
        s = s[np.lexsort(s.T[::-1])]
        assert np.array_equal(orc.delaunay(P), s)


@pytest.mark.parametrize("D,n,kind", [(2, 20000, "uniform"), (2, 20000, "normal"),
                                      (3, 5000, "uniform"), (3, 5000, "clustered")])
def test_euler_hull_and_volume(orc, D, n, kind):
    spatial = pytest.importorskip("scipy.spatial")
    if kind == "uniform":
        P = pointsets.uniform(n, D, 31)
    elif kind == "normal":
        P = pointsets.normal(n, D, 31)
    else:
        P = pointsets.clustered(n, 31)
    a = orc.delaunay(P)
    c = orc.check_combinatorics(a, n)
    hull = spatial.ConvexHull(P)
    assert c["h"] == len(hull.vertices)
    orc.check_volume(P, a, hull.volume)


@pytest.mark.parametrize("D,n", [(2, 3000), (3, 1500)])
def test_locally_delaunay(orc, D, n):
    P = pointsets.uniform(n, D, 41)
    a = orc.delaunay(P)
    assert orc.check_locally_delaunay(P, a) > 0


def test_errors(orc):
    P = pointsets.uniform(50, 2, 1)
    P[7] = P[3]
    with pytest.raises(orc.OracleError, match="duplicate"):
        orc.delaunay(P)
    L = np.stack([np.arange(10.0), 2 * np.arange(10.0)], axis=1)
    with pytest.raises(orc.OracleError, match="degenerate"):
        orc.delaunay(L)
    Q = np.concatenate([pointsets.uniform(30, 2, 3), np.zeros((30, 1))], axis=1)
    with pytest.raises(orc.OracleError, match="degenerate"):
        orc.delaunay(Q)


def test_nearest_matches_numpy(orc):
    rng = np.random.default_rng(8)
    S = rng.random((200, 3))
    Q = rng.random((2000, 3))
    d = ((Q[:, None, :] - S[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(orc.nearest(Q, S), np.argmin(d, axis=1))
    # exact ties resolve to the smaller rank
    S2 = np.array([[0.0, 0.0], [2.0, 0.0], [1.0, 5.0]])
    Q2 = np.array([[1.0, 0.0]])
    assert orc.nearest(Q2, S2)[0] == 0
    assert orc.nearest(Q2, S2, np.array([5, 1, 0]))[0] == 1


# ---------------------------------------------------------------- neighbour relation
def py_neighbors(S):
    """Quadratic definition: rows r, t are neighbours across r's j-th vertex
    when they share every vertex of r but that one."""
    S = [list(map(int, r)) for r in S]
    out = [[-1] * len(r) for r in S]
    for r, a in enumerate(S):
        for t, b in enumerate(S):
            if t == r:
                continue
            common = set(a) & set(b)
            if len(common) == len(a) - 1:
                j = [x for x in a if x not in common][0]
                out[r][a.index(j)] = t
    return np.array(out, dtype=np.int64).reshape(-1, len(S[0]) if S else 1)


@pytest.mark.parametrize("D,n,shape", [(2, 40, "uniform"), (2, 36, "grid"), (3, 30, "uniform"), (3, 27, "grid")])
def test_neighbors_match_quadratic_definition(orc, D, n, shape):
    P = pointsets.uniform(n, D, 5) if shape == "uniform" else pointsets.grid((6, 6) if D == 2 else (3, 3, 3), seed=5)
    S = orc.delaunay(P)
    assert np.array_equal(orc.neighbors(S), py_neighbors(S))


@pytest.mark.parametrize("D,n", [(2, 3000), (3, 2000)])
def test_neighbors_hull_count_and_symmetry(orc, D, n):
    spatial = pytest.importorskip("scipy.spatial")
    P = pointsets.uniform(n, D, 77)
    S = orc.delaunay(P)
    N = orc.neighbors(S)
    h = len(spatial.ConvexHull(P).vertices)
    hull_facets = int((N < 0).sum())
    assert hull_facets == (h if D == 2 else 2 * h - 4)
    r, j = np.nonzero(N >= 0)
    t = N[r, j]
    assert np.all((N[t] == r[:, None]).sum(axis=1) == 1)      # the link is returned exactly once
    # the two rows share all but one vertex
    shared = (S[r][:, :, None] == S[t][:, None, :]).any(axis=2).sum(axis=1)
    assert np.all(shared == D)


def test_neighbors_reject_a_facet_in_three_rows(orc):
    S = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]])
    with pytest.raises(AssertionError):
        orc.neighbors(S)
