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
