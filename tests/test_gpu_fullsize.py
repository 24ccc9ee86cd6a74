"""GPU parity at the full workload sizes, in the launch configuration the
benchmark times.

* 1,000,000 uniform 3D points, k = 16, 0.5 % sample: the whole output is
  compared element by element with the oracle's DT (integer output:
  bit-exact), for the sample divide, the kd median divide and recursive
  bisection.
* 4,000,000 clustered 3D points, k = 64, 0.5 % sample: the whole output is
  compared element by element with the oracle's DT (a few minutes of one
  host core), for the sample divide and the kd divide; the device
  certificate (local Delaunay, hull convexity, Euler characteristic, every
  point a vertex) and an exact empty-sphere check of sampled simplices run
  beside it as independent checks.
"""
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


def test_uniform3d_1m_k16_matches_oracle(tri):
    P = pointsets.workload("uniform3d_1m")
    want = oracle.delaunay(P)
    got = tri.triangulate(P, k=16, sample_frac=0.005).astype(np.int64)
    st = tri.stats()
    assert st.k == 16 and st.border_vertices > 0
    assert np.array_equal(got, want)
    tri.configure(divide=1)
    try:
        kd = tri.triangulate(P, k=16, sample_frac=0.005).astype(np.int64)
    finally:
        tri.configure(divide=0)
    assert np.array_equal(kd, want)
    tri.configure(recursive=1)
    try:
        rb = tri.triangulate(P, k=16, sample_frac=0.005).astype(np.int64)
        assert tri.stats().k == 16
    finally:
        tri.configure(recursive=0)
    assert np.array_equal(rb, want)


def _empty_sphere_sample(P, S, m, seed):
    """Checks m random simplices of S one by one: no point of P lies inside
    the perturbed circumsphere (exact oracle predicates on every point within
    the FP64 circumball enlarged by 10 %)."""
    spatial = pytest.importorskip("scipy.spatial")
    tree = spatial.cKDTree(P)
    rng = np.random.default_rng(seed)
    rows = S[rng.choice(len(S), m, replace=False)]
    tuples = []
    for r in rows:
        A = P[r]
        M = 2.0 * (A[1:] - A[0])
        b = (A[1:] ** 2).sum(1) - (A[0] ** 2).sum()
        c = np.linalg.solve(M, b)
        rad = np.sqrt(((A - c) ** 2).sum(1)).max()
        near = tree.query_ball_point(c, rad * 1.1 + 1e-12)     # every point near the sphere, tested exactly
        v = [int(x) for x in r]                  # the oracle normalises the orientation
        for q in near:
            if q not in v:
                tuples.append(v + [q])
    if tuples:
        T = np.array(tuples, dtype=np.int32)
        assert np.all(oracle.predicates(P, "insphere", T) < 0)
    return len(tuples)


def test_clustered3d_4m_k64_matches_oracle(tri):
    P = pointsets.workload("clustered3d_4m")
    tri.configure(validate=1, neighbors=1)
    try:
        S = tri.triangulate(P, k=64, sample_frac=0.005).astype(np.int64)
        st = tri.stats()
    finally:
        tri.configure(validate=0, neighbors=0)
    assert st.k == 64 and st.validated == 1 and st.border_vertices > 0
    tri.configure(divide=1)
    try:
        kd = tri.triangulate(P, k=64, sample_frac=0.005).astype(np.int64)
    finally:
        tri.configure(divide=0)
    want = oracle.delaunay(P)
    assert np.array_equal(S, want)
    assert np.array_equal(kd, want)
    assert _empty_sphere_sample(P, S, 300, 5) > 0
