"""The autotuner's search on the host: every candidate timed, the fastest
applied, the report sorted (a stand-in binding and timer, no GPU)."""
from paper_1512_02831_gb300 import tune


class FakeBinding:
    class BkdError(RuntimeError):
        pass

    def __init__(self, screen: bool, cost):
        self.screen = screen
        self.cost = cost       # options -> seconds
        self.opts = {}
        self.queries = 0

    def bkd_set_option(self, tree, key, val):
        if key == "precision" and val == 1 and not self.screen:
            raise self.BkdError("no screen data")
        self.opts[key] = val

    def bkd_query(self, tree, Q, k):
        self.queries += 1


def fake_timer(binding):
    return lambda run: (run(), binding.cost(dict(binding.opts)))[1]


def test_picks_the_fastest_and_applies_it():
    cost = lambda o: (1.0 if o["precision"] == 0 else 0.4) + \
        abs(o["tail_queries"] - 8192) * 1e-6
    b = FakeBinding(True, cost)
    rep = tune.autotune("tree", "Q", 10, tails=(0, 8192, 32768), repeats=3,
                        timer=fake_timer(b), bkd=b)
    assert rep["best"] == {"precision": 1, "tail_queries": 8192}
    assert b.opts == rep["best"]
    times = [t for _, t in rep["timings"]]
    assert times == sorted(times) and len(times) == 6
    # each candidate: one warm-up + `repeats` timed calls
    assert b.queries == 6 * (1 + 3)


def test_without_screen_data_only_float32_candidates():
    b = FakeBinding(False, lambda o: o["tail_queries"] * 1e-6 + 1.0)
    rep = tune.autotune("tree", "Q", 5, tails=(2048, 0), timer=fake_timer(b),
                        bkd=b)
    assert all(o["precision"] == 0 for o, _ in rep["timings"])
    assert rep["best"] == {"precision": 0, "tail_queries": 0}
    assert tune.candidates(False, (1, 2)) == [
        {"precision": 0, "tail_queries": 1},
        {"precision": 0, "tail_queries": 2}]
