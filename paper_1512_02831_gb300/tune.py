"""Autotuning of the schedule and launch-shape options of a tree.

Times ``bkd_query`` on a caller-supplied query sample and leaves the tree on
the fastest setting of the options that change only how the work is laid
out -- leaf scoring (float32 / BF16 screen), the screen kernel (warp /
tcgen05, when the tree holds both layouts), the tail threshold, the queries
per screened work item, the rounds queued per host look and the screen's
CTAs per SM.  Results do not depend on any of them (the tests assert bit
equality across them), so tuning never changes an answer.  A candidate the
tree rejects (a screen kernel whose layout it lacks, an item size outside
the selected kernel's range) is skipped.

The search is coordinate-wise: the options are taken one after the other,
every candidate value of the current option is timed with the others at
their best values so far, and the fastest is kept; `sweeps` passes repeat
that.  Each timing is the best of `repeats` calls after a warm-up call.

    report = autotune(tree, Q_sample, k)
    report["best"]      # the options now set on the tree
"""
from __future__ import annotations

import time

# option -> candidate values, in search order (the first value of each is
# the starting point)
SPACE = {
    "precision": (1, 0),
    "screen_kernel": (0, 1),
    "tail_queries": (-1, 0, 2048, 8192, 32768, 65536),
    # the warp kernel takes 8..32, the tcgen05 kernel 16..128
    "screen_tile": (32, 24, 16, 128, 96, 64),
    "round_batch": (0, 1, 4, 16, 64),
    "screen_ctas": (0, 1, 2),
}
SCREEN_ONLY = ("screen_kernel", "screen_tile", "screen_ctas")


def _wall_timer(run) -> float:
    """Seconds of one synchronous call (bkd_query returns when done)."""
    t0 = time.perf_counter()
    run()
    return time.perf_counter() - t0


def space_for(screen_available: bool, space=None) -> dict:
    """The search space without the screen's options when the tree has no
    screen data."""
    space = dict(SPACE if space is None else space)
    if not screen_available:
        space["precision"] = (0,)
        for key in SCREEN_ONLY:
            space.pop(key, None)
    return space


def autotune(tree, Q, k: int, screen_available: bool | None = None,
             space=None, sweeps: int = 1, repeats: int = 2, timer=None,
             bkd=None) -> dict:
    """Coordinate search over `space` (default SPACE); applies the fastest
    setting to `tree` and returns {"best": options, "timings": [(options,
    seconds), ...] in the order timed, "calls": bkd_query calls made}.
    `screen_available`: whether the tree was built with precision=1 (None:
    probe by setting it).  `timer(run) -> seconds` and `bkd` (the binding
    module) can be replaced, e.g. in tests."""
    if bkd is None:
        import paper_1512_02831_gb300 as bkd
    timer = timer or _wall_timer
    if screen_available is None:
        try:
            bkd.bkd_set_option(tree, "precision", 1)
            screen_available = True
        except bkd.BkdError:
            screen_available = False
    space = space_for(screen_available, space)
    best = {key: vals[0] for key, vals in space.items()}
    cache = {}
    timings = []
    calls = 0

    def measure(opts):
        nonlocal calls
        key = tuple(sorted(opts.items()))
        if key in cache:
            return cache[key]
        try:
            for name, val in opts.items():
                bkd.bkd_set_option(tree, name, val)
        except bkd.BkdError:
            cache[key] = float("inf")  # not valid on this tree
            return cache[key]
        bkd.bkd_query(tree, Q, k)  # warm-up (workspace, caches)
        calls += 1
        sec = min(timer(lambda: bkd.bkd_query(tree, Q, k))
                  for _ in range(max(1, repeats)))
        calls += max(1, repeats)
        cache[key] = sec
        timings.append((dict(opts), sec))
        return sec

    for _ in range(max(1, sweeps)):
        for name, vals in space.items():
            if name in SCREEN_ONLY and best.get("precision") == 0:
                continue  # no screened rounds to shape
            scores = {v: measure(dict(best, **{name: v})) for v in vals}
            best[name] = min(scores, key=scores.get)
            if name == "screen_kernel":
                # the item size resets with the kernel: restart its search
                # from the kernel's default
                best["screen_tile"] = 32 if best[name] == 0 else 128
    for name, val in best.items():
        bkd.bkd_set_option(tree, name, val)
    return {"best": best, "timings": timings, "calls": calls,
            "best_seconds": cache[tuple(sorted(best.items()))]}
