"""GPU parity of the merge's neighbourhood update and of the Delaunay
certificate (dt_get_neighbors, dt_validate, dt_config.validate).

Neighbours are compared element by element with the oracle's definition
(integer output: bit-exact).  The certificate must pass the oracle's DT and
flag triangulations that were made wrong on the CPU (a flipped edge, a
missing or repeated simplex, a bad index, an unused point)."""
import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tri():
    from paper_1902_07554_gb300 import Triangulator
    t = Triangulator(0)
    yield t
    t.close()


CASES = [
    ("uniform2d", lambda: pointsets.uniform(20_000, 2, 3), 4, 0.01),
    ("normal2d", lambda: pointsets.normal(12_000, 2, 4), 1, 0.0),
    ("grid2d", lambda: pointsets.grid((90, 70), seed=5), 4, 0.02),
    ("uniform3d", lambda: pointsets.uniform(30_000, 3, 6), 8, 0.005),
    ("clustered3d", lambda: pointsets.clustered(30_000, 7), 8, 0.005),
    ("grid3d", lambda: pointsets.grid((16, 14, 12), seed=8), 4, 0.02),
    ("uniform3d_direct", lambda: pointsets.uniform(8_000, 3, 9), 1, 0.0),
]


@pytest.mark.parametrize("name,make,k,frac", CASES, ids=[c[0] for c in CASES])
def test_neighbors_match_oracle(tri, name, make, k, frac):
    P = make()
    tri.configure(base_threshold=256)
    try:
        S = tri.triangulate(P, k=k, sample_frac=frac).astype(np.int64)
        N = tri.neighbors().astype(np.int64)
    finally:
        tri.configure(base_threshold=2048, validate=0, neighbors=0)
    want = oracle.delaunay(P)
    assert np.array_equal(S, want)
    assert np.array_equal(N, oracle.neighbors(want))
    assert tri.stats().hull_facets == int((N < 0).sum())


@pytest.mark.parametrize("dim", [2, 3])
def test_validate_inside_the_pipeline(tri, dim):
    P = pointsets.uniform(40_000, dim, 10 + dim)
    tri.configure(validate=1, neighbors=1, base_threshold=256)
    try:
        S = tri.triangulate(P, k=8, sample_frac=0.005)
        st = tri.stats()
    finally:
        tri.configure(base_threshold=2048, validate=0, neighbors=0)
    assert st.validated == 1 and st.ms_phase[7] > 0
    assert np.array_equal(S.astype(np.int64), oracle.delaunay(P))


@pytest.mark.parametrize("dim", [2, 3])
def test_certificate_accepts_the_oracle(tri, dim):
    P = pointsets.uniform(5_000, dim, 20 + dim)
    S = oracle.delaunay(P)
    v = tri.validate(P, S[np.random.default_rng(1).permutation(len(S))][:, ::-1])   # any row order / tuple order
    assert v["violations"] == 0, v
    assert v["simplices"] == len(S) and v["euler"] == 1
    assert v["edges"] == len(oracle.edges(S))
    N = oracle.neighbors(S)
    assert v["hull_facets"] == int((N < 0).sum())
    assert v["interior_facets"] == int((N >= 0).sum()) // 2


def _flip_one_edge_2d(P, S):
    """Replace two triangles sharing an interior edge whose quadrilateral is
    strictly convex by the other diagonal (a valid but non-Delaunay triangulation)."""
    N = oracle.neighbors(S)
    for r in range(len(S)):
        for j in range(3):
            t = N[r, j]
            if t <= r:
                continue
            a = S[r, j]
            e = [x for x in S[r] if x != a]
            b = [x for x in S[t] if x not in e][0]
            def orient(p, q, s):
                return np.sign((P[q, 0] - P[p, 0]) * (P[s, 1] - P[p, 1]) - (P[q, 1] - P[p, 1]) * (P[s, 0] - P[p, 0]))
            # convex: a and b on opposite sides of e, e's endpoints on opposite sides of ab
            if orient(e[0], e[1], a) * orient(e[0], e[1], b) < 0 and orient(a, b, e[0]) * orient(a, b, e[1]) < 0:
                T = np.delete(S, [r, t], axis=0)
                return np.concatenate([T, np.sort([[a, b, e[0]], [a, b, e[1]]], axis=1)])
    raise AssertionError("no flippable edge")


def test_certificate_rejects_wrong_triangulations(tri):
    P = pointsets.uniform(2_000, 2, 31)
    S = oracle.delaunay(P)
    v = tri.validate(P, _flip_one_edge_2d(P, S))
    assert v["non_delaunay"] >= 1 and v["violations"] >= 1, v
    v = tri.validate(P, S[1:])                        # a hole or a dent
    assert v["violations"] >= 1, v
    v = tri.validate(P, np.concatenate([S, S[:1]]))   # a repeated simplex
    assert v["violations"] >= 1, v
    bad = S.copy()
    bad[5, 1] = len(P) + 3                            # index out of range
    v = tri.validate(P, bad)
    assert v["bad_index"] == 1 and v["violations"] >= 1, v
    sub = oracle.delaunay(P[:-1])                     # the last point is no vertex
    v = tri.validate(P, sub)
    assert v["unused_points"] == 1, v
    Q = P.copy()
    Q[:, 0] *= -1.0                                   # a mirror image keeps every circumcircle empty
    assert tri.validate(Q, S)["violations"] == 0


def test_certificate_rejects_a_3d_triangulation_of_moved_points(tri):
    P = pointsets.uniform(3_000, 3, 41)
    S = oracle.delaunay(P)
    Q = P.copy()
    Q[100] = Q[100] + 0.05                           # the old triangulation is no longer Delaunay for Q
    v = tri.validate(Q, S)
    assert v["violations"] >= 1, v
    assert tri.validate(Q, oracle.delaunay(Q))["violations"] == 0


def test_neighbors_unavailable_after_a_batch(tri):
    from paper_1902_07554_gb300 import DTError
    P = pointsets.uniform(500, 2, 1)
    tri.triangulate_batch(P, np.array([0, 250, 500]))
    with pytest.raises(DTError, match="ARG"):
        tri.neighbors()
