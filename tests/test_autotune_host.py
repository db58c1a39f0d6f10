"""The plan autotuner's bookkeeping (no GPU): exploration hands out every
candidate, exploitation picks the fastest per workload class, and the state
survives a JSON round trip."""
from paper_2606_20441_b300 import autotune, inputs


class FakeHandle:
    def __init__(self):
        self.tuning = None

    def pp_set_tuning(self, g, h, tile_caps=(0, 0, 0, 0)):
        self.tuning = (g, h) + tuple(c for c in tile_caps[:2] if c)


def test_explore_then_exploit_per_class():
    cands = [(16, 1.6), (8, 1.6), (32, 2.0), (0, 0.0, 200, 448)]
    speed = {(16, 1.6): 5.0, (8, 1.6): 3.0, (32, 2.0): 9.0, (0, 0.0, 200, 448): 7.0}
    t = autotune.Tuner(cands, trials=2)
    rng = inputs.SplitMix64(7)
    a = inputs.random_tfim(rng, "a", 4, 4, 5, 5, 1e-4, w_max=8)
    b = inputs.random_tfim(rng, "b", 8, 8, 20, 20, 1e-5, w_max=10)
    assert autotune.class_key(a) != autotune.class_key(b)
    h = FakeHandle()
    seen = []
    for _ in range(len(cands) * 2):
        s = t.apply(h, a)
        assert h.tuning == s
        seen.append(s)
        t.observe(a, s, updates=speed[s] * 1e9, seconds=1.0)
    assert sorted(seen) == sorted(cands * 2)
    for _ in range(3):
        assert t.apply(h, a) == (32, 2.0)
    # the other class starts its own exploration
    assert t.apply(h, b) == cands[0]
    t2 = autotune.Tuner.from_json(t.to_json(), cands)
    assert t2.best(autotune.class_key(a)) == (32, 2.0)
    assert t2.choose(autotune.class_key(a)) == (32, 2.0)
    assert t2.samples[autotune.class_key(a)][(0, 0.0, 200, 448)] == [7.0e9, 7.0e9]


def test_failed_runs_are_not_scored():
    t = autotune.Tuner([(16, 1.6), (8, 1.6)], trials=1)
    rng = inputs.SplitMix64(9)
    a = inputs.random_tfim(rng, "a", 4, 4, 5, 5, 1e-4)
    t.observe(a, (8, 1.6), updates=0.0, seconds=1.0)
    t.observe(a, (16, 1.6), updates=1e9, seconds=1.0)
    assert t.best(autotune.class_key(a)) == (16, 1.6)
