"""GPU parity: device predicates and the direct (k = 1) triangulation against
the CPU oracle, element by element (integer output: bit-exact)."""
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


def _tuples(rng, n, w, m):
    return np.array([rng.choice(n, w, replace=False) for _ in range(m)], dtype=np.int32)


@pytest.mark.parametrize("D", [2, 3])
def test_predicates_random(tri, D):
    rng = np.random.default_rng(1 + D)
    P = rng.random((200, D))
    for kind, w in [("orient", D + 1), ("insphere_raw", D + 2), ("insphere", D + 2), ("closer", 3)]:
        T = _tuples(rng, 200, w, 2000)
        assert np.array_equal(tri.eval_predicates(P, kind, T), oracle.predicates(P, kind, T)), kind


@pytest.mark.parametrize("D", [2, 3])
def test_predicates_degenerate_and_near_degenerate(tri, D):
    rng = np.random.default_rng(7)
    base = pointsets.grid((4,) * D) * 0.1 + 0.3
    gid = rng.permutation(len(base)).astype(np.int64)
    for trial in range(4):
        P = base.copy()
        if trial:
            idx = rng.choice(len(P), 5, replace=False)
            for i in idx:
                c = rng.integers(D)
                P[i, c] = np.nextafter(P[i, c], np.inf if rng.random() < 0.5 else -np.inf)
        for kind, w in [("orient", D + 1), ("insphere_raw", D + 2), ("insphere", D + 2), ("closer", 3)]:
            T = _tuples(rng, len(P), w, 3000)
            assert np.array_equal(tri.eval_predicates(P, kind, T, gid), oracle.predicates(P, kind, T, gid)), kind
    assert tri.stats().exact_calls > 0


@pytest.mark.parametrize("D", [2, 3])
def test_predicates_near_the_fp32_bound(tri, D):
    """Tuples whose determinants sit near the FP32 stage's error bound:
    cospherical points moved by relative amounts from 1e-9 to 1e-4, and a
    tight cluster beside one far outlier (a large eta for every test)."""
    rng = np.random.default_rng(11 + D)
    u = rng.normal(size=(300, D))
    S = 0.3 * u / np.linalg.norm(u, axis=1, keepdims=True) + 0.5
    S *= 1.0 + 10.0 ** rng.uniform(-9, -4, size=(300, 1)) * rng.choice([-1, 1], size=(300, 1))
    C = np.concatenate([0.5 + 1e-3 * rng.random((199, D)), np.full((1, D), 900.0)])
    for P in (S, C):
        for kind, w in [("orient", D + 1), ("insphere_raw", D + 2), ("insphere", D + 2)]:
            T = _tuples(rng, len(P) - (P is C), w, 4000)
            assert np.array_equal(tri.eval_predicates(P, kind, T), oracle.predicates(P, kind, T)), kind


def test_predicates_wide_exponent_range(tri):
    P = np.array([[1e-200, 0.0], [1.0, 1e-150], [0.0, 1.0], [1.0, 1.0], [1e100, 1e-100], [3e-5, 7e-9]])
    rng = np.random.default_rng(0)
    for kind, w in [("orient", 3), ("insphere_raw", 4), ("closer", 3)]:
        T = _tuples(rng, 6, w, 300)
        try:
            got = tri.eval_predicates(P, kind, T)
        except Exception as e:            # the exact path may report DT_E_RANGE; never a wrong sign
            assert "RANGE" in str(e)
            continue
        assert np.array_equal(got, oracle.predicates(P, kind, T)), kind


@pytest.mark.parametrize("D,n,kind", [(2, 10, "uniform"), (2, 1000, "uniform"), (2, 20000, "normal"),
                                      (3, 12, "uniform"), (3, 1000, "uniform"), (3, 20000, "clustered")])
def test_direct_dt_matches_oracle(tri, D, n, kind):
    if kind == "uniform":
        P = pointsets.uniform(n, D, 5)
    elif kind == "normal":
        P = pointsets.normal(n, D, 5)
    else:
        P = pointsets.clustered(n, 5)
    got = tri.triangulate(P, k=1)
    assert got.dtype == np.int32
    assert np.array_equal(got.astype(np.int64), oracle.delaunay(P))
    assert tri.stats().simplices == len(got)


@pytest.mark.parametrize("shape", [(7, 5), (12, 12), (4, 4, 4), (5, 3, 2), (6, 6, 6)])
def test_direct_dt_degenerate_grids(tri, shape):
    P = pointsets.grid(shape, seed=3)
    got = tri.triangulate(P, k=1)
    assert np.array_equal(got.astype(np.int64), oracle.delaunay(P))


def test_direct_dt_cocircular(tri):
    P = pointsets.cocircular(20, 2)
    got = tri.triangulate(P, k=1)
    assert np.array_equal(got.astype(np.int64), oracle.delaunay(P))


def test_errors(tri):
    from paper_1902_07554_gb300 import DTError
    P = pointsets.uniform(100, 2, 1)
    P[10] = P[20]
    with pytest.raises(DTError, match="DUPLICATE"):
        tri.triangulate(P)
    L = np.stack([np.arange(50.0), 3 * np.arange(50.0)], axis=1)
    with pytest.raises(DTError, match="DEGENERATE"):
        tri.triangulate(L)
    Q = pointsets.uniform(50, 3, 2)
    Q[:, 2] = 0.5
    with pytest.raises(DTError, match="DEGENERATE"):
        tri.triangulate(Q)
    bad = pointsets.uniform(10, 2, 1)
    bad[3, 1] = np.nan
    with pytest.raises(DTError, match="ARG"):
        tri.triangulate(bad)
    # the context stays usable after errors
    P = pointsets.uniform(500, 2, 9)
    assert np.array_equal(tri.triangulate(P).astype(np.int64), oracle.delaunay(P))


@pytest.mark.parametrize("D,k", [(2, 1), (2, 4), (3, 1), (3, 8)])
def test_large_region_path_matches_oracle(tri, D, k):
    """Tiny regular region lists (cavity_cap = 8) send most regions through the
    large-region pass (grown again with the pass bit in their key); the
    result must still be the oracle's DT."""
    P = pointsets.clustered(20_000, 9) if D == 3 else pointsets.normal(20_000, 2, 9)
    tri.configure(cavity_cap=8, base_threshold=256)
    try:
        got = tri.triangulate(P, k=k, sample_frac=0.01).astype(np.int64)
    finally:
        tri.configure(cavity_cap=0, base_threshold=2048)
    assert np.array_equal(got, oracle.delaunay(P))


@pytest.mark.parametrize("D,kind", [(2, "uniform"), (3, "clustered")])
def test_single_block_rounds_match_oracle(tri, D, kind):
    """Every round inside one thread block (small_rounds above n) and none
    there (small_rounds = -1) give the oracle's DT."""
    P = pointsets.clustered(6_000, 13) if kind == "clustered" else pointsets.uniform(6_000, D, 13)
    want = oracle.delaunay(P)
    for sr in (1_000_000, -1):
        tri.configure(small_rounds=sr)
        try:
            got = tri.triangulate(P, k=1).astype(np.int64)
        finally:
            tri.configure(small_rounds=0)
        assert np.array_equal(got, want), sr


@pytest.mark.parametrize("cfg", [dict(cavity_occupancy=12), dict(cavity_occupancy=16), dict(cavity_group=16),
                                 dict(nominate_rings=2, cavity_blocks=8), dict(active_ratio=25)])
def test_schedule_knobs_match_oracle(tri, cfg):
    """Launch shapes and schedules change which nominees win a round, never
    the result: each gives the oracle's DT (plain path and 4 partitions)."""
    P = pointsets.clustered(30_000, 21)
    want = oracle.delaunay(P)
    tri.configure(**cfg)
    try:
        for k in (1, 4):
            assert np.array_equal(tri.triangulate(P, k=k, sample_frac=0.01).astype(np.int64), want), (cfg, k)
    finally:
        tri.configure(**{name: 0 for name in cfg})
