"""Pins for the divide / border / merge references (Alg. 1 and Alg. 2).

The strongest pin: running the paper's merge (Alg. 1 (border triangulation and merging)) on the
exact border set reproduces DT(P) exactly, for sample-based and kd labels,
and stays exact when the border set is enlarged arbitrarily (a conservative
intersection primitive only ever adds simplices).
"""
import itertools
import math

import numpy as np
import pytest

import pointsets
from oracle import divide as dv


def test_splitmix64_published_vector():
    # First output of SplitMix64 seeded with 0 (published reference value).
    assert dv.splitmix64(0) == 0xE220A8397B1DCDAF


def test_sample_ids_definition():
    n, eta = 5000, 50
    s = dv.sample_ids(n, eta, 7)
    assert len(s) == eta and len(np.unique(s)) == eta and np.all(np.diff(s) > 0)
    assert s.min() >= 0 and s.max() < n
    # different seeds give different samples; same seed the same
    assert not np.array_equal(s, dv.sample_ids(n, eta, 8))
    assert np.array_equal(s, dv.sample_ids(n, eta, 7))
    assert dv.sample_size(10000, 0.01, 2) == 100
    assert dv.sample_size(10000, 0.0, 3) == 100
    assert dv.sample_size(10, 0.01, 3) == 5


def test_sample_is_roughly_uniform():
    n = 4000
    hits = np.zeros(n)
    for seed in range(200):
        hits[dv.sample_ids(n, 40, seed)] += 1
    # each index is drawn with probability 40/4000 per seed -> mean 2
    assert abs(hits.mean() - 2.0) < 1e-9
    assert hits[: n // 2].sum() / hits.sum() == pytest.approx(0.5, abs=0.05)


@pytest.mark.parametrize("bits,D", [(3, 2), (2, 3), (4, 2)])
def test_hilbert_key_is_a_hilbert_curve(bits, D):
    """Keys form a permutation of the cells and consecutive cells are face
    neighbours (the defining property of a Hilbert curve)."""
    cells = list(itertools.product(range(1 << bits), repeat=D))
    keys = [dv.hilbert_key(np.array(c), bits) for c in cells]
    assert sorted(keys) == list(range(len(cells)))
    order = [c for _, c in sorted(zip(keys, cells))]
    for a, b in zip(order, order[1:]):
        assert sum(abs(x - y) for x, y in zip(a, b)) == 1


def test_graph_is_sample_dt_edges(orc):
    P = pointsets.uniform(2000, 2, 3)
    ids = dv.sample_ids(2000, 60, 1)
    E, w = dv.sample_graph(P[ids], ids)
    T = orc.bruteforce(P[ids])
    assert np.array_equal(E, orc.edges(T))
    h = orc.hull_vertex_count(T)
    assert len(E) == 3 * 60 - 3 - h
    # Table 1 log weight: -ln(|v-w| / d*), scaled by 1000, at least 1
    PS = P[ids]
    dstar = np.linalg.norm(PS.max(0) - PS.min(0))
    d = np.linalg.norm(PS[E[:, 0]] - PS[E[:, 1]], axis=1) / dstar
    assert np.all(np.abs(w - np.maximum(1, np.rint(-1000 * np.log(d)))) == 0)
    assert np.all(w >= 1)


@pytest.mark.parametrize("init", ["hilbert", "kd"])
@pytest.mark.parametrize("D,k", [(2, 4), (2, 7), (3, 16)])
def test_partition_balance_and_cut(orc, D, k, init):
    P = pointsets.clustered(3000, 5) if D == 3 else pointsets.normal(3000, 2, 5)
    ids = dv.sample_ids(3000, 400, 2)
    PS = P[ids]
    E, w = dv.sample_graph(PS, ids)
    b0 = dv.partition(PS, E, w, k, rounds=0, init=init)
    b = dv.partition(PS, E, w, k, init=init)
    lmin, lmax = dv.partition_bounds(400, k, 0.05)
    sizes = np.bincount(b, minlength=k)
    assert sizes.max() <= lmax and sizes.min() >= lmin
    assert dv.cut_weight(E, w, b) <= dv.cut_weight(E, w, b0)
    assert np.array_equal(b, dv.partition(PS, E, w, k, init=init))
    if init == "kd":
        # before refinement: the median boxes of the sample, sizes within one
        assert np.array_equal(b0, dv.kd_labels(PS, k))
        s0 = np.bincount(b0, minlength=k)
        assert s0.max() - s0.min() <= 1


def test_partition_initial_blocks_by_hand():
    """Eight points on a line, k = 2, no refinement: Hilbert runs and the kd
    median split both put the four leftmost points in block 0."""
    PS = np.array([[x, 0.1 * (x % 2)] for x in (5, 1, 7, 3, 0, 6, 2, 4)], dtype=np.float64)
    E = np.zeros((0, 2), dtype=np.int64)
    w = np.zeros(0, dtype=np.int64)
    want = (PS[:, 0] >= 4).astype(np.int64)
    assert np.array_equal(dv.partition(PS, E, w, 2, rounds=0, init="kd"), want)
    assert np.array_equal(dv.partition(PS, E, w, 2, rounds=0, init="hilbert"), want)


def test_kd_labels_are_median_boxes():
    P = pointsets.clustered(1000, 9)
    lab = dv.kd_labels(P, 8)
    sizes = np.bincount(lab, minlength=8)
    assert sizes.max() - sizes.min() <= 1
    # first split on x: leaves 0-3 lie left of leaves 4-7
    assert P[lab < 4, 0].max() <= P[lab >= 4, 0].min()
    assert P[lab < 2, 1].max() <= P[(lab >= 2) & (lab < 4), 1].min()
    lab5 = dv.kd_labels(P, 5)
    assert np.bincount(lab5).sum() == 1000 and len(np.unique(lab5)) == 5


def test_labels_are_nearest_sample_block():
    P = pointsets.uniform(3000, 3, 4)
    ids = dv.sample_ids(3000, 80, 3)
    block = np.arange(80) % 5
    lab = dv.labels(P, P[ids], ids, block)
    d = ((P[:, None, :] - P[ids][None, :, :]) ** 2).sum(-1)
    assert np.array_equal(lab, block[np.argmin(d, axis=1)])
    assert np.all(lab[ids] == block)


def test_metrics_values():
    m = dv.metrics(np.array([90, 110, 100, 100]), 400, 10, 30)
    assert m["imbalance"] == pytest.approx(0.1)
    assert m["min_deviation"] == pytest.approx(-0.1)
    assert m["cv"] == pytest.approx(math.sqrt(200 / 3) / 100)
    assert m["o_dt"] == pytest.approx(440 / 400)


def _sample_labels(P, k, frac, seed):
    n, D = P.shape
    eta = dv.sample_size(n, frac, D)
    ids = dv.sample_ids(n, eta, seed)
    E, w = dv.sample_graph(P[ids], ids)
    block = dv.partition(P[ids], E, w, k)
    return dv.labels(P, P[ids], ids, block)


@pytest.mark.parametrize("D,n,k,kind", [(2, 400, 4, "sample"), (2, 300, 5, "kd"),
                                        (3, 160, 3, "sample"), (3, 160, 4, "kd")])
def test_divide_and_conquer_reproduces_dt(orc, D, n, k, kind):
    P = pointsets.uniform(n, D, 17) if D == 2 else pointsets.clustered(n, 17)
    lab = _sample_labels(P, k, 0.1, 3) if kind == "sample" else dv.kd_labels(P, k)
    Bset, VB, parts = dv.border_exact(P, lab, k)
    assert 0 < len(VB) < n
    T = dv.merge(parts, Bset, VB, P, lab)
    assert np.array_equal(T, orc.delaunay(P))


def test_merge_is_exact_for_any_border_superset(orc):
    P = pointsets.normal(300, 2, 23)
    lab = dv.kd_labels(P, 4)
    Bset, VB, parts = dv.border_exact(P, lab, 4)
    rng = np.random.default_rng(0)
    want = orc.delaunay(P)
    for trial in range(3):
        B2 = set(Bset)
        for ids, T, _ in parts:
            pick = rng.random(len(T)) < 0.15
            B2.update(tuple(int(x) for x in s) for s in T[pick])
        VB2 = np.array(sorted(set(VB.tolist()) | {x for s in B2 for x in s}), dtype=np.int64)
        assert np.array_equal(dv.merge(parts, B2, VB2, P, lab), want)


def test_degenerate_partition_contributes_all_points(orc):
    """A partition holding only collinear points cannot be triangulated; all
    of its points join the border set and the merge stays exact."""
    P = pointsets.uniform(120, 2, 2)
    line = np.stack([np.linspace(0.1, 0.9, 6), np.full(6, 0.123456)], axis=1)
    P = np.vstack([P, line])
    lab = np.zeros(len(P), dtype=np.int64)
    lab[P[:, 0] > 0.5] = 1
    lab[120:] = 2
    Bset, VB, parts = dv.border_exact(P, lab, 3)
    assert set(range(120, 126)) <= set(VB.tolist())
    assert np.array_equal(dv.merge(parts, Bset, VB, P, lab), orc.delaunay(P))


def test_recursive_labels_first_level_is_the_direct_bisection():
    """Depth 0 of recursive bisection is Alg. 2 with k = 2 on all points: the
    leaves of k = 8 fall on the sides of the k = 2 split."""
    P = pointsets.uniform(3000, 2, 23)
    direct = _sample_labels(P, 2, 0.02, 5)
    assert np.array_equal(dv.recursive_labels(P, 2, 0.02, 5), direct)
    lab8 = dv.recursive_labels(P, 8, 0.02, 5)
    assert np.array_equal(lab8 >= 4, direct == 1)
    sizes = np.bincount(lab8, minlength=8)
    assert sizes.sum() == 3000 and sizes.min() > 0
    # the second level splits each half on its own fresh sample
    left = np.nonzero(direct == 0)[0]
    eta = dv.sample_size(len(left), 0.02, 2)
    sids = dv.sample_ids(len(left), eta, 6)
    E, w = dv.sample_graph(P[left][sids], sids)
    side = dv.labels(P[left], P[left][sids], sids, dv.partition(P[left][sids], E, w, 2))
    assert np.array_equal(lab8[left] >= 2, side == 1)
    with pytest.raises(ValueError):
        dv.recursive_labels(P, 6, 0.02, 5)


@pytest.mark.parametrize("D,n,k,kind", [(2, 600, 4, "sample"), (2, 500, 8, "kd"), (3, 240, 4, "sample"),
                                        (3, 200, 4, "kd")])
def test_recursive_merges_reproduce_dt(orc, D, n, k, kind):
    """k - 1 pairwise merges (Sec. 3.1) reach DT(P), and every node's border is
    non-empty."""
    P = pointsets.uniform(n, D, 29) if D == 2 else pointsets.clustered(n, 29)
    lab = dv.recursive_labels(P, k, 0.1, 4) if kind == "sample" else dv.kd_labels(P, k)
    rows, sizes = dv.recursive_merges(P, lab, k)
    assert sum(len(level) for level in sizes) == k - 1
    assert [len(level) for level in sizes] == [k >> h for h in range(1, k.bit_length())]
    assert all(x > 0 for level in sizes for x in level)
    assert np.array_equal(rows, orc.delaunay(P))


@pytest.mark.parametrize("kind,want", [("log", [511, 223, 1]), ("constant", [1, 1, 1]),
                                       ("inverse", [1667, 1250, 1000]), ("linear", [400, 200, 1])])
def test_table1_weights_by_hand(kind, want):
    """Table 1 on a 3-4-5 triangle: d* = 5 (the box diagonal), so the edges have
    d = 0.6, 0.8, 1.0; weights are 1000 omega rounded, at least 1 (-ln 0.6 =
    0.5108, -ln 0.8 = 0.2231, 1/0.6 = 1.6667)."""
    PS = np.array([[0.0, 0.0], [3.0, 0.0], [0.0, 4.0]])
    E = np.array([[0, 1], [0, 2], [1, 2]])
    assert dv.edge_weights(PS, E, kind).tolist() == want


@pytest.mark.parametrize("shape,k", [((24, 20), 4), ((8, 7, 6), 2)])
def test_recursive_merges_on_a_lattice(orc, shape, k):
    """Maximally degenerate input (cocircular / cospherical lattice points):
    the perturbed predicates keep the k - 1 merges exact."""
    P = pointsets.grid(shape, seed=3)
    lab = dv.kd_labels(P, k)
    rows, sizes = dv.recursive_merges(P, lab, k)
    assert np.array_equal(rows, orc.delaunay(P))
    assert sum(len(level) for level in sizes) == k - 1


def test_bfs_border_equals_the_sweep_on_connected_partitions():
    """Alg. 1's hull-seeded breadth-first search reaches the same exact border
    set as testing every simplex when the partitions have no islands."""
    P = pointsets.uniform(1500, 2, 1)
    lab = _sample_labels(P, 4, 0.05, 1)
    B1, V1, _ = dv.border_exact(P, lab, 4)
    B2, V2, _ = dv.border_exact_bfs(P, lab, 4)
    assert B1 == B2 and np.array_equal(V1, V2)


def test_bfs_border_misses_an_island(orc):
    """A partition enclosed by another (an island, which unions of Voronoi
    cells allow): the simplices of the outer partition that span the island
    are border simplices unreachable from its hull, so the breadth-first
    search misses them and the merge is wrong; testing every simplex (the
    GPU's sweep) keeps it exact."""
    P = pointsets.uniform(800, 2, 11)
    lab = (np.linalg.norm(P - 0.5, axis=1) < 0.15).astype(np.int64)
    want = orc.delaunay(P)
    B1, V1, parts = dv.border_exact(P, lab, 2)
    B2, V2, _ = dv.border_exact_bfs(P, lab, 2)
    assert B2 < B1
    assert np.array_equal(dv.merge(parts, B1, V1, P, lab), want)
    assert not np.array_equal(dv.merge(parts, B2, V2, P, lab), want)


def _golden_partition():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "partition_lp_ml.txt")
    g = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        g[key] = vals
    return g


def _edges_of(vals):
    t = np.array([int(x) for x in vals], dtype=np.int64).reshape(-1, 3)
    return t[:, :2], t[:, 2]


def test_lp_refine_hand_derived_rounds():
    """Tie-break (smaller block), parity of the moving vertices, and the
    acceptance order (earlier candidates counted whether accepted or not)
    against a case worked out on paper (tests/golden/partition_lp_ml.txt)."""
    g = _golden_partition()
    n, k, eps = int(g["lp.n"][0]), int(g["lp.k"][0]), float(g["lp.eps"][0])
    E, w = _edges_of(g["lp.edges"])
    lmin, lmax = dv.partition_bounds(n, k, eps)
    assert (lmin, lmax) == (2, 4)
    nbrs = dv.adjacency(n, E, w)
    init = np.array([int(x) for x in g["lp.init"]])
    one = dv.lp_refine(nbrs, [1] * n, init, k, lmin, lmax, 1)
    two = dv.lp_refine(nbrs, [1] * n, init, k, lmin, lmax, 2)
    assert one.tolist() == [int(x) for x in g["lp.after1"]]
    assert two.tolist() == [int(x) for x in g["lp.after2"]]


def test_multilevel_hand_derived_case():
    """Heavy-edge matching, contraction and the coarse move of a bound pair
    that single-vertex moves cannot make (tests/golden/partition_lp_ml.txt)."""
    g = _golden_partition()
    n, k, eps = int(g["ml.n"][0]), int(g["ml.k"][0]), float(g["ml.eps"][0])
    E, w = _edges_of(g["ml.edges"])
    PS = np.stack([np.arange(n, dtype=np.float64), np.zeros(n)], axis=1)
    assert dv.partition(PS, E, w, k, eps, rounds=2).tolist() == [int(x) for x in g["ml.lp2"]]
    tr = {}
    got = dv.ml_partition(PS, E, w, k, eps, rounds=2, trace=tr, coarse_rounds=2)
    assert tr["sizes"] == [8, 4]
    assert tr["mates"][0].tolist() == [int(x) for x in g["ml.mate"]]
    assert tr["cmaps"][0].tolist() == [int(x) for x in g["ml.cmap"]]
    cnbrs, cvw = tr["coarse"][0]
    assert cvw == [2, 2, 2, 2]
    ce = sorted((a, b, ww) for a in range(4) for b, ww in cnbrs[a] if a < b)
    want = [int(x) for x in g["ml.coarse_edges"]]
    assert ce == [tuple(want[i:i + 3]) for i in range(0, len(want), 3)]
    assert tr["refined"][0].tolist() == [int(x) for x in g["ml.coarse_refined"]]
    assert got.tolist() == [int(x) for x in g["ml.result"]]
    assert dv.cut_weight(E, w, got) == 1 and dv.cut_weight(E, w, dv.partition(PS, E, w, k, eps, rounds=2)) == 20


@pytest.mark.parametrize("k,init", [(4, "kd"), (16, "kd"), (16, "hilbert")])
def test_multilevel_invariants(k, init):
    """On a sample graph: every block weight within [lmin, lmax] at the end,
    every coarse level a contraction of the one below (vertex weights sum to
    eta, coarse vertices at most cmax), and a cut no heavier than the
    initial blocks'."""
    P = pointsets.clustered(60_000, 5)
    ids = dv.sample_ids(len(P), 1200, 3)
    PS = P[ids]
    E, w = dv.sample_graph(PS, ids)
    lmin, lmax = dv.partition_bounds(len(PS), k, 0.05)
    tr = {}
    b = dv.ml_partition(PS, E, w, k, 0.05, rounds=8, init=init, trace=tr)
    sizes = np.bincount(b, minlength=k)
    assert sizes.min() >= lmin and sizes.max() <= lmax
    assert len(tr["sizes"]) >= 2 and all(a > b2 for a, b2 in zip(tr["sizes"], tr["sizes"][1:]))
    for _, cvw in tr["coarse"]:
        assert sum(cvw) == len(PS) and max(cvw) <= max(2, lmax // 4)
    assert dv.cut_weight(E, w, b) <= dv.cut_weight(E, w, dv.initial_blocks(PS, k, init))


def test_lp_refine_counts_rejected_candidates():
    """A rejected candidate still counts against its target's room
    (tests/golden/partition_lp_ml.txt, case LP2)."""
    g = _golden_partition()
    n, k, eps = int(g["lp2.n"][0]), int(g["lp2.k"][0]), float(g["lp2.eps"][0])
    E, w = _edges_of(g["lp2.edges"])
    lmin, lmax = dv.partition_bounds(n, k, eps)
    assert (lmin, lmax) == (3, 5)
    init = np.array([int(x) for x in g["lp2.init"]])
    got = dv.lp_refine(dv.adjacency(n, E, w), [1] * n, init, k, lmin, lmax, 1)
    assert got.tolist() == [int(x) for x in g["lp2.after1"]]


def test_matching_hand_derived():
    """Handshake matching: ties to the smaller neighbour, no pair across
    blocks, the weight cap (tests/golden/partition_lp_ml.txt, case M)."""
    g = _golden_partition()
    n = int(g["m.n"][0])
    E, w = _edges_of(g["m.edges"])
    block = np.array([int(x) for x in g["m.block"]])
    nbrs = dv.adjacency(n, E, w)
    cmax = int(g["m.cmax"][0])
    assert dv.match_heavy_edges(nbrs, [1] * n, block, cmax, 4).tolist() == [int(x) for x in g["m.mate_unit"]]
    vw = [int(x) for x in g["m.weights"]]
    assert dv.match_heavy_edges(nbrs, vw, block, cmax, 4).tolist() == [int(x) for x in g["m.mate_weighted"]]
