"""The seeded input generators: a batch instance generated alone equals its
slice of the whole batch (the all-core CPU baseline relies on it)."""
import numpy as np

import pointsets


def test_batch_instance_alone_equals_its_slice():
    P, off, kinds = pointsets.batch_instances(count=96, seed=4)
    for i in (0, 1, 47, 95):
        Q = pointsets.batch_instance(i, count=96, seed=4)
        assert np.array_equal(Q, P[off[i]:off[i + 1]])
    assert {"uniform", "normal"} <= set(kinds)


def test_generators_are_seeded_and_in_range():
    for make in (lambda s: pointsets.uniform(5000, 3, s), lambda s: pointsets.normal(5000, 2, s),
                 lambda s: pointsets.clustered(5000, s)):
        a, b, c = make(1), make(1), make(2)
        assert np.array_equal(a, b) and not np.array_equal(a, c)
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        assert len(np.unique(a, axis=0)) == len(a)          # no duplicate points
    U = pointsets.uniform(5000, 3, 1)
    assert U.min() >= 0.0 and U.max() < 1.0


def test_clustered_recipe():
    """Blob points inside the unit cube, heightfield points within 0.4 (+ noise)
    of z = 0.5, and a very uneven density."""
    P = pointsets.clustered(20_000, 7)
    assert P.shape == (20_000, 3)
    assert np.all(P[:, :2] >= 0.0) and np.all(P[:, :2] <= 1.0)
    # blob points lie inside the cube; surface points within 8 x 0.05 (+ noise) of z = 0.5
    inside = np.all((P >= 0.0) & (P <= 1.0), axis=1)
    assert inside.mean() > 0.99
    # the blobs make the density very uneven: the fullest of 1000 cells holds far more than 20
    cells = np.floor(np.clip(P, 0, 1 - 1e-12) * 10).astype(int)
    counts = np.bincount(cells[:, 0] * 100 + cells[:, 1] * 10 + cells[:, 2], minlength=1000)
    assert counts.max() > 20 * 10


def test_cocircular_points_are_exactly_on_the_circle():
    C = pointsets.cocircular(12, 1)
    assert len(C) == 12 and np.all(C[:, 0] ** 2 + C[:, 1] ** 2 == 625.0)


def test_serving_jobs_recipe():
    sizes, kinds, seeds = pointsets.serve_jobs(2000, seed=5)
    assert sizes.min() >= 1000 and sizes.max() <= 2_000_000
    assert set(kinds) == {"uniform", "clustered"}
    logs = np.log(sizes)
    assert abs(logs.mean() - (np.log(1000) + np.log(2_000_000)) / 2) < 0.2   # log-uniform
