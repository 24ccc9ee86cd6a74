"""GPU parity for the divide-and-conquer path (Alg. 1 + Alg. 2).

The final triangulation is exact, so it must equal the oracle's DT(P)
bit for bit for every k, divide, primitive and seed (k-invariance).  The
divide sub-steps are compared with the oracle's references: sample indices
(bit-exact), sample blocks (bit-exact, integer weights), labels (bit-exact,
exact nearest-site), and the border vertex set must contain the exact one.
"""
import numpy as np
import pytest

import oracle
import pointsets
from oracle import divide as dv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tri():
    from paper_1902_07554_gb300 import Triangulator
    t = Triangulator(0, base_threshold=16)
    yield t
    t.close()


def _cfg(tri, **kw):
    base = dict(divide=0, primitive=0, weight=0, lp_rounds=16, epsilon=0.05, grid_cell=1.0, seed=1,
                base_threshold=16, validate=0, cavity_cap=0, recursive=0, partition_init=0, partitioner=0)
    base.update(kw)
    tri.configure(**base)


def test_uniform2d_10k_k4_matches_oracle(tri):
    """2D, 10,000 uniform points, k = 4 from a 1% sample."""
    _cfg(tri)
    P = pointsets.workload("uniform2d_10k")
    got = tri.triangulate(P, k=4, sample_frac=0.01)
    assert np.array_equal(got.astype(np.int64), oracle.delaunay(P))
    s = tri.stats()
    assert s.k == 4 and s.eta == 100 and 0 < s.border_vertices < 10000


@pytest.mark.parametrize("D,n,kind", [(2, 30000, "normal"), (3, 20000, "uniform"), (3, 30000, "clustered")])
@pytest.mark.parametrize("k", [2, 7, 16])
def test_k_invariance_sample_divide(tri, D, n, kind, k):
    P = {"uniform": lambda: pointsets.uniform(n, D, 11), "normal": lambda: pointsets.normal(n, D, 11),
         "clustered": lambda: pointsets.clustered(n, 11)}[kind]()
    _cfg(tri)
    want = oracle.delaunay(P)
    got = tri.triangulate(P, k=k, sample_frac=0.01)
    assert np.array_equal(got.astype(np.int64), want)


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("divide,prim", [(0, 1), (1, 0), (1, 1), (0, 2), (1, 2)])
def test_k_invariance_divides_and_primitives(tri, D, divide, prim):
    P = pointsets.clustered(20000, 5) if D == 3 else pointsets.normal(20000, 2, 5)
    want = oracle.delaunay(P)
    _cfg(tri, divide=divide, primitive=prim)
    for k in (4, 16):
        got = tri.triangulate(P, k=k, sample_frac=0.005)
        assert np.array_equal(got.astype(np.int64), want), (k, divide, prim)


@pytest.mark.parametrize("seed", [1, 2, 99])
def test_sample_seed_and_weight_invariance(tri, seed):
    P = pointsets.uniform(20000, 3, 8)
    want = oracle.delaunay(P)
    for w in (0, 1, 2, 3):
        _cfg(tri, seed=seed, weight=w)
        got = tri.triangulate(P, k=8, sample_frac=0.01)
        assert np.array_equal(got.astype(np.int64), want), (seed, w)


def test_degenerate_grid_with_partitions(tri):
    P = pointsets.grid((30, 30), seed=4)
    want = oracle.delaunay(P)
    _cfg(tri)
    for k in (2, 4, 9):
        got = tri.triangulate(P, k=k, sample_frac=0.05)
        assert np.array_equal(got.astype(np.int64), want)
    P3 = pointsets.grid((12, 12, 12), seed=4)
    want3 = oracle.delaunay(P3)
    for k in (2, 8):
        got = tri.triangulate(P3, k=k, sample_frac=0.05)
        assert np.array_equal(got.astype(np.int64), want3)


@pytest.mark.parametrize("D,n,k,frac", [(2, 10000, 4, 0.01), (3, 20000, 16, 0.005)])
def test_divide_steps_match_oracle(tri, D, n, k, frac):
    P = pointsets.uniform(n, D, 3) if D == 2 else pointsets.clustered(n, 3)
    _cfg(tri, seed=7)
    tri.triangulate(P, k=k, sample_frac=frac)
    eta = dv.sample_size(n, frac, D)
    ids = dv.sample_ids(n, eta, 7)
    assert np.array_equal(tri.sample().astype(np.int64), ids)
    E, w = dv.sample_graph(P[ids], ids)
    block = dv.partition(P[ids], E, w, k)
    assert np.array_equal(tri.sample_blocks().astype(np.int64), block)
    lab = dv.labels(P, P[ids], ids, block)
    assert np.array_equal(tri.labels().astype(np.int64), lab)
    s = tri.stats()
    sizes = np.bincount(lab, minlength=k)
    m = dv.metrics(sizes, n, eta, s.border_vertices)
    assert s.imbalance == pytest.approx(m["imbalance"]) and s.cv == pytest.approx(m["cv"])
    assert s.cut_weight == dv.cut_weight(E, w, block)


def test_kd_labels_match_oracle(tri):
    P = pointsets.clustered(20000, 6)
    _cfg(tri, divide=1)
    for k in (8, 5):
        tri.triangulate(P, k=k)
        assert np.array_equal(tri.labels().astype(np.int64), dv.kd_labels(P, k))


@pytest.mark.parametrize("D,n,k", [(2, 1500, 4), (3, 600, 3)])
def test_border_vertices_contain_exact_border(tri, D, n, k):
    P = pointsets.uniform(n, D, 21)
    counts = {}
    for prim in (0, 2):
        _cfg(tri, divide=1, primitive=prim)
        tri.triangulate(P, k=k)
        lab = tri.labels().astype(np.int64)
        assert np.array_equal(lab, dv.kd_labels(P, k))
        _, VB, _ = dv.border_exact(P, lab, k)
        got = set(tri.border_vertices().tolist())
        assert set(VB.tolist()) <= got, prim
        assert len(got) < n
        counts[prim] = len(got)
    assert counts[2] <= counts[0]          # the points are a subset of their cells


def test_label_points_entry(tri):
    rng = np.random.default_rng(3)
    S = rng.random((300, 3))
    Q = rng.random((20000, 3))
    srank = rng.permutation(300).astype(np.int64)
    block = rng.integers(0, 9, size=300).astype(np.int32)
    got = tri.label_points(Q, S, srank, block)
    want = block[oracle.nearest(Q, S, srank)]
    assert np.array_equal(got, want)


def test_partition_graph_entry(tri):
    P = pointsets.normal(5000, 2, 12)
    ids = dv.sample_ids(5000, 500, 3)
    E, w = dv.sample_graph(P[ids], ids)
    for k in (3, 8, 16):
        got = tri.partition_graph(P[ids], E, w, k, 0.05, 16)
        assert np.array_equal(got.astype(np.int64), dv.partition(P[ids], E, w, k, init="kd"))
    tri.configure(partition_init="hilbert")
    try:
        for k in (3, 8):
            got = tri.partition_graph(P[ids], E, w, k, 0.05, 16)
            assert np.array_equal(got.astype(np.int64), dv.partition(P[ids], E, w, k, init="hilbert"))
    finally:
        tri.configure(partition_init="auto")


@pytest.mark.parametrize("gen,D,eta,k,init", [("normal", 2, 500, 3, "kd"), ("normal", 2, 500, 16, "kd"),
                                               ("clustered", 3, 3000, 64, "kd"), ("uniform", 3, 2000, 16, "hilbert"),
                                               ("clustered", 3, 20000, 64, "kd")])
def test_multilevel_partition_matches_oracle(tri, gen, D, eta, k, init):
    """The multilevel partitioner (matchings inside the blocks, contraction,
    weighted label propagation on every level) gives the oracle's blocks bit
    for bit, down to the full 0.5 % sample of the 4M clustered workload."""
    n = eta * 100 if gen != "normal" else 5000
    P = {"normal": lambda: pointsets.normal(n, D, 12), "uniform": lambda: pointsets.uniform(n, D, 5),
         "clustered": lambda: pointsets.clustered(n, 7)}[gen]()
    ids = dv.sample_ids(len(P), eta, 3)
    E, w = dv.sample_graph(P[ids], ids)
    _cfg(tri, partitioner=1, partition_init=init)
    try:
        got = tri.partition_graph(P[ids], E, w, k, 0.05, 16).astype(np.int64)
    finally:
        _cfg(tri, partitioner=0, partition_init="auto")
    want = dv.ml_partition(P[ids], E, w, k, 0.05, 16, init=init)
    assert np.array_equal(got, want)
    lmin, lmax = dv.partition_bounds(eta, k, 0.05)
    sizes = np.bincount(got, minlength=k)
    assert sizes.min() >= lmin and sizes.max() <= lmax


@pytest.mark.parametrize("D,n,k,frac,divide", [(2, 20000, 4, 0.01, 0), (2, 20000, 8, 0.01, 1),
                                               (3, 20000, 8, 0.005, 0), (3, 16000, 4, 0.01, 1)])
def test_recursive_bisection_matches_oracle(tri, D, n, k, frac, divide):
    P = pointsets.uniform(n, D, 31) if D == 2 else pointsets.clustered(n, 31)
    want = oracle.delaunay(P)
    _cfg(tri, recursive=1, divide=divide, base_threshold=256)
    got = tri.triangulate(P, k=k, sample_frac=frac).astype(np.int64)
    st = tri.stats()
    lab = tri.labels().astype(np.int64)
    N = tri.neighbors().astype(np.int64)
    assert np.array_equal(got, want)
    assert np.array_equal(N, oracle.neighbors(want))
    assert st.k == k and st.border_vertices > 0 and st.border_dt_simplices > 0
    ref = dv.recursive_labels(P, k, frac, 1) if divide == 0 else dv.kd_labels(P, k)
    assert np.array_equal(lab, ref)
    if divide == 0:   # one fresh sample per node: k - 1 samples
        L = k.bit_length() - 1
        eta = sum(dv.sample_size(int(m), frac, D) for t in range(L) for m in np.bincount(lab >> (L - t)) if m)
        assert st.eta == eta


@pytest.mark.parametrize("D,n,k,divide", [(2, 1200, 4, 0), (3, 500, 4, 1)])
def test_recursive_border_contains_exact_borders(tri, D, n, k, divide):
    """Per merge the grid border is a superset of the exact one, so the
    levels' border vertex counts add up to at least the exact counts."""
    P = pointsets.uniform(n, D, 33)
    _cfg(tri, recursive=1, divide=divide, base_threshold=16)
    got = tri.triangulate(P, k=k, sample_frac=0.1).astype(np.int64)
    st = tri.stats()
    lab = tri.labels().astype(np.int64)
    rows, sizes = dv.recursive_merges(P, lab, k)
    assert np.array_equal(got, rows)
    assert st.border_vertices >= sum(sum(level) for level in sizes)
    bv = set(tri.border_vertices().tolist())
    for h in range(1, k.bit_length()):
        part = lab >> (h - 1)
        for v in range(len(sizes[h - 1])):
            ids = np.nonzero((part >> 1) == v)[0]
            _, VB, _ = dv.border_exact(P[ids], part[ids] & 1, 2)
            assert set(ids[VB].tolist()) <= bv


def test_recursive_bisection_needs_a_power_of_two(tri):
    from paper_1902_07554_gb300 import DTError
    P = pointsets.uniform(5000, 2, 2)
    _cfg(tri, recursive=1, base_threshold=256)
    with pytest.raises(DTError, match="ARG"):
        tri.triangulate(P, k=6)
    assert np.array_equal(tri.triangulate(P, k=1).astype(np.int64), oracle.delaunay(P))
