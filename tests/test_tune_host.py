"""Host logic of the schedule autotuner (tune.py) with a stand-in context
and a stand-in clock: every candidate is timed, the fastest is applied and
remembered per workload shape.  No GPU."""
import numpy as np

from paper_1902_07554_gb300 import tune


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeTri:
    """Each call advances the clock by a cost that depends on the schedule."""

    def __init__(self, clock, best):
        self.clock, self.best, self.cfg, self.calls = clock, best, {}, []

    def configure(self, **cfg):
        self.cfg.update(cfg)

    def _cost(self):
        d = sum(abs(self.cfg.get(k, 0) - v) for k, v in self.best.items())
        return 0.010 + 1e-5 * d

    def triangulate(self, P, k=1, sample_frac=0.0, fetch=True):
        self.calls.append(("single", dict(self.cfg)))
        self.clock.t += self._cost()

    def triangulate_batch(self, P, off, fetch=True):
        self.calls.append(("batch", dict(self.cfg)))
        self.clock.t += self._cost()


def test_picks_and_applies_the_fastest_schedule():
    tune.clear_cache()
    clk = FakeClock()
    best = {"brio_growth": 200, "brio_drain": 4, "cavity_blocks": 8, "first_batch": 128, "nominate_rings": 2}
    tri = FakeTri(clk, best)
    P = np.zeros((1000, 3))
    r = tune.autotune(tri, P, k=1, clock=clk)
    assert r["best"] == best and not r["cached"]
    assert tri.cfg == best
    assert len(r["table"]) == len(tune.candidates()) == 48   # 3 x 2 x 2 x 2 x 2
    assert len(tri.calls) == 48 * 3                      # one untimed + two timed runs each
    assert abs(r["ms"] - 10.0) < 1e-9
    # the same shape again: applied from the cache, nothing timed
    tri.cfg = {}
    r2 = tune.autotune(tri, np.ones((1000, 3)), k=1, clock=clk)
    assert r2["cached"] and tri.cfg == best and len(tri.calls) == 48 * 3


def test_batch_shapes_and_ties():
    tune.clear_cache()
    clk = FakeClock()
    tri = FakeTri(clk, {})                               # every schedule costs the same
    P = np.zeros((5000, 2))
    off = np.array([0, 1000, 2500, 5000])
    grid = {"brio_drain": (2, 8), "brio_growth": (150,)}
    r = tune.autotune(tri, P, offsets=off, grid=grid, reps=1, clock=clk)
    assert r["best"] == tune.candidates(grid)[0]           # ties go to the first candidate
    assert all(kind == "batch" for kind, _ in tri.calls)
    assert tune.shape_key(P, off) == (2, 2, 11, 1)
    assert tune.shape_key(P, off) != tune.shape_key(P)     # a batch is another shape
