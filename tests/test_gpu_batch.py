"""GPU parity of the batched form: many independent instances in one engine
run, each bit-identical to the oracle's DT of that instance."""
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


def _mixed(count, seed, lo, hi, dim=2):
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    parts = []
    for i, m in enumerate(sizes):
        r = np.random.default_rng(seed * 1000 + i)
        parts.append(r.random((m, dim)) if r.random() < 0.5 else r.normal(0.5, 0.1, size=(m, dim)))
    off = np.zeros(count + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return np.concatenate(parts), off


@pytest.mark.parametrize("dim", [2, 3])
def test_batch_matches_oracle_per_instance(tri, dim):
    P, off = _mixed(60, 3 + dim, 4, 3000, dim)
    res = tri.triangulate_batch(P, off)
    st = tri.batch_status(len(off) - 1)
    for i in range(len(off) - 1):
        Q = P[off[i]:off[i + 1]]
        if len(Q) <= dim:
            assert st[i] != 0 and len(res[i]) == 0
            continue
        assert st[i] == 0
        assert np.array_equal(res[i].astype(np.int64), oracle.delaunay(Q)), i


def test_batch_degenerate_and_tiny_instances(tri):
    a = pointsets.uniform(300, 2, 1)
    line = np.stack([np.arange(20.0), np.arange(20.0) * 0.5], axis=1)
    tiny = np.array([[0.0, 0.0], [1.0, 0.0]])
    grid = pointsets.grid((9, 7), seed=2)
    P = np.concatenate([a, line, tiny, grid, a])          # the same points again in another instance: allowed
    off = np.array([0, 300, 320, 322, 385, 685], dtype=np.int64)
    res = tri.triangulate_batch(P, off)
    st = tri.batch_status(5)
    assert list(st) == [0, -3, -1, 0, 0]
    assert len(res[1]) == 0 and len(res[2]) == 0
    assert np.array_equal(res[0].astype(np.int64), oracle.delaunay(a))
    assert np.array_equal(res[4].astype(np.int64), oracle.delaunay(a))
    assert np.array_equal(res[3].astype(np.int64), oracle.delaunay(grid))


def test_batch_rejects_duplicates_inside_an_instance(tri):
    from paper_1902_07554_gb300 import DTError
    a = pointsets.uniform(100, 2, 4)
    a[50] = a[7]
    with pytest.raises(DTError, match="DUPLICATE"):
        tri.triangulate_batch(a, np.array([0, 100]))


def _oracle_digests(job):
    """Worker (spawned process): the oracle's DT of the given batch instances,
    each as (index, SHA-1 of its int64 canonical array, row count)."""
    import hashlib

    import oracle as orc
    import pointsets as ps
    ids, count, seed = job
    out = []
    for i in ids:
        T = orc.delaunay(ps.batch_instance(int(i), count=count, seed=seed)).astype(np.int64)
        out.append((int(i), hashlib.sha1(np.ascontiguousarray(T).tobytes()).hexdigest(), len(T)))
    return out


def test_batch2d_4096_full_size_every_instance(tri):
    """The full batched workload (4,096 instances, 256..65,536 points each,
    uniform or normal by instance seed, 49.5M points) in one call: every
    instance equals the oracle's DT of that instance.  The oracle runs on
    every host core (spawned processes, each generating its own instances);
    results are compared through SHA-1 digests of the canonical int64 arrays,
    and a mismatching instance is recomputed here and compared in full."""
    import hashlib
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    P, off, kinds = pointsets.batch_instances()
    res = tri.triangulate_batch(P, off)
    assert len(res) == 4096
    cores = max(1, min(os.cpu_count() or 1, 32))
    order = np.argsort(-(off[1:] - off[:-1]))              # largest first, dealt round robin
    shares = [(order[c::cores], 4096, 4) for c in range(cores)]
    with ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as ex:
        digests = [d for part in ex.map(_oracle_digests, shares) for d in part]
    assert len(digests) == 4096
    bad = []
    for i, dig, rows in digests:
        got = np.ascontiguousarray(res[i].astype(np.int64))
        if len(got) != rows or hashlib.sha1(got.tobytes()).hexdigest() != dig:
            bad.append(i)
    for i in bad[:3]:
        assert np.array_equal(res[i].astype(np.int64), oracle.delaunay(P[off[i]:off[i + 1]])), i
    assert not bad, bad[:20]


def test_autotuned_schedule_keeps_parity(tri):
    """The autotuner times every candidate schedule (round schedule, nominee
    queue, cavity tiles) on a batch and applies the fastest; the batch
    triangulated under it equals the oracle instance by instance."""
    from paper_1902_07554_gb300 import tune
    P, off = _mixed(80, 17, 200, 6000)
    tune.clear_cache()
    r = tune.autotune(tri, P, offsets=off, reps=1, use_cache=False)
    assert len(r["table"]) == len(tune.candidates()) and set(r["best"]) == set(tune.DEFAULT_GRID)
    res = tri.triangulate_batch(P, off)
    try:
        for i in range(len(off) - 1):
            assert np.array_equal(res[i].astype(np.int64), oracle.delaunay(P[off[i]:off[i + 1]])), i
    finally:
        tri.configure(**{k: 0 for k in tune.DEFAULT_GRID})
