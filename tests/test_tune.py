"""The autotuner's search on the host: every candidate timed, the fastest
applied, the report sorted (a stand-in binding and timer, no GPU)."""
from paper_1512_02831_gb300 import tune


class FakeBinding:
    class BkdError(RuntimeError):
        pass

    def __init__(self, screen: bool, cost, kernels=(0, 1)):
        self.screen = screen
        self.kernels = kernels  # screen kernels whose layout the tree holds
        self.cost = cost       # options -> seconds
        self.opts = {"screen_kernel": kernels[0] if kernels else 0}
        self.queries = 0

    def bkd_set_option(self, tree, key, val):
        # the library's rules: screen data needed for precision 1, the
        # kernel's layout for screen_kernel, the kernel's item-size range
        # for screen_tile, and the item size resets with the kernel
        if key == "precision" and val == 1 and not self.screen:
            raise self.BkdError("no screen data")
        if key == "screen_kernel":
            if val not in self.kernels:
                raise self.BkdError("no layout")
            if val != self.opts.get("screen_kernel"):
                self.opts["screen_tile"] = 32 if val == 0 else 128
        if key == "screen_tile":
            lo, hi = (8, 32) if self.opts.get("screen_kernel") == 0 else (16, 128)
            if not (lo <= val <= hi and val % lo == 0):
                raise self.BkdError("item size out of range")
        self.opts[key] = val

    def bkd_query(self, tree, Q, k):
        self.queries += 1


def fake_timer(binding):
    return lambda run: (run(), binding.cost(dict(binding.opts)))[1]


def separable_cost(o):
    """A cost whose optimum is known: each option contributes on its own."""
    return ((1.0 if o["precision"] == 0 else 0.4)
            + (0.0 if o.get("screen_kernel", 0) == 1 else 0.1)
            + abs(o["tail_queries"] - 8192) * 1e-6
            + (0.0 if o.get("screen_tile", 128) == 64 else 0.05)
            + (0.0 if o.get("round_batch", 0) == 16 else 0.02)
            + (0.0 if o.get("screen_ctas", 0) == 0 else 0.01))


def test_coordinate_search_finds_the_separable_optimum_and_applies_it():
    b = FakeBinding(True, separable_cost)
    rep = tune.autotune("tree", "Q", 10, repeats=3, timer=fake_timer(b),
                        bkd=b)
    want = {"precision": 1, "screen_kernel": 1, "tail_queries": 8192,
            "screen_tile": 64, "round_batch": 16, "screen_ctas": 0}
    assert rep["best"] == want
    assert b.opts == want
    assert rep["best_seconds"] == min(t for _, t in rep["timings"])
    # every distinct valid setting timed once: one warm-up + `repeats`
    # calls each; rejected candidates cost no call
    assert b.queries == rep["calls"] == len(rep["timings"]) * (1 + 3)
    assert len(rep["timings"]) < 2 * 2 * 6 * 6 * 5 * 3  # not the full grid


def test_candidates_the_tree_rejects_are_skipped():
    """A tree with the warp kernel's layout only: the tcgen05 kernel and
    item sizes above 32 are rejected by the library and never timed."""
    b = FakeBinding(True, separable_cost, kernels=(0,))
    rep = tune.autotune("tree", "Q", 10, timer=fake_timer(b), bkd=b)
    assert rep["best"]["screen_kernel"] == 0
    assert rep["best"]["screen_tile"] in (8, 16, 24, 32)
    assert all(o["screen_kernel"] == 0 and o["screen_tile"] <= 32
               for o, _ in rep["timings"])


def test_without_screen_data_only_float32_and_no_screen_shapes():
    b = FakeBinding(False, lambda o: abs(o["tail_queries"]) * 1e-6 + 1.0)
    rep = tune.autotune("tree", "Q", 5, timer=fake_timer(b), bkd=b)
    assert all(o["precision"] == 0 for o, _ in rep["timings"])
    assert all("screen_tile" not in o and "screen_ctas" not in o
               and "screen_kernel" not in o for o, _ in rep["timings"])
    assert rep["best"]["tail_queries"] == 0
    assert "screen_tile" not in tune.space_for(False)


def test_a_second_sweep_can_improve_a_coupled_cost():
    """Coupled options: the best tail depends on the round batch; a second
    sweep revisits the tail with the round batch found in the first."""
    def cost(o):
        rb = o.get("round_batch", 0)
        return (abs(o["tail_queries"] - (32768 if rb == 64 else 2048)) * 1e-6
                + (0.0 if rb == 64 else 0.05) + (o["precision"] == 0))
    b = FakeBinding(True, cost)
    one = tune.autotune("t", "Q", 1, sweeps=1, timer=fake_timer(b), bkd=b)
    two = tune.autotune("t", "Q", 1, sweeps=2, timer=fake_timer(b), bkd=b)
    assert two["best_seconds"] <= one["best_seconds"]
    assert two["best"]["tail_queries"] == 32768
