"""Device loop limits run out on purpose, with no GPU fault: every device
wait and walk in the insertion engine has an iteration limit after which the
kernel records an error status and returns.  Configured tiny, each limit must
end the call with its error code (DT_E_TIMEOUT for the round and walk limits,
DT_E_OVERFLOW for a simplex arena that stays too small through its retries),
and the same context must then produce the oracle's triangulation."""
import numpy as np
import pytest

import oracle
import pointsets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tri():
    from paper_1902_07554_gb300 import Triangulator
    t = Triangulator(0, base_threshold=256)
    yield t
    t.close()


def _fails_then_recovers(tri, P, k, code, **limits):
    from paper_1902_07554_gb300 import DTError
    tri.configure(**limits)
    try:
        with pytest.raises(DTError) as e:
            tri.triangulate(P, k=k, sample_frac=0.02)
        assert e.value.code == code, e.value
    finally:
        tri.configure(**{key: 0 for key in limits})
    got = tri.triangulate(P, k=k, sample_frac=0.02).astype(np.int64)
    assert np.array_equal(got, oracle.delaunay(P))


@pytest.mark.parametrize("dim,k", [(2, 1), (3, 1), (3, 4)])
def test_round_limit_times_out_then_context_recovers(tri, dim, k):
    P = pointsets.uniform(6000, dim, 40 + dim)
    _fails_then_recovers(tri, P, k, -5, round_limit=3)


@pytest.mark.parametrize("dim", [2, 3])
def test_walk_limit_times_out_then_context_recovers(tri, dim):
    P = pointsets.uniform(6000, dim, 50 + dim)
    _fails_then_recovers(tri, P, 1, -5, walk_limit=1)


def test_small_arena_overflows_then_context_recovers(tri):
    # one slot per point, doubled three times: 8 per point, far below the
    # ~27 a 3D insertion run allocates (dead slots are not reused)
    P = pointsets.uniform(6000, 3, 61)
    _fails_then_recovers(tri, P, 1, -6, arena_factor=1)


def test_limits_in_the_batched_form(tri):
    from paper_1902_07554_gb300 import DTError
    Q = pointsets.uniform(3000, 2, 7)
    off = np.array([0, 1000, 3000])
    tri.configure(round_limit=2)
    try:
        with pytest.raises(DTError):
            tri.triangulate_batch(Q, off)
    finally:
        tri.configure(round_limit=0)
    res = tri.triangulate_batch(Q, off)
    for i in range(2):
        assert np.array_equal(res[i].astype(np.int64), oracle.delaunay(Q[off[i]:off[i + 1]]))
