"""Autotuning of the run-time options of a tree.

Times ``bkd_query`` on a caller-supplied query sample under each candidate
setting of the options that change only the schedule -- leaf scoring
(float32 / BF16 screen) and the tail threshold -- and leaves the tree on the
fastest.  Results do not depend on these options (the tests assert bit
equality across them), so tuning never changes an answer.

    report = autotune(tree, Q_sample, k)
    report["best"]      # the options now set on the tree
"""
from __future__ import annotations

import itertools
import time

DEFAULT_TAILS = (0, 2048, 8192, 32768, 65536)


def candidates(screen_available: bool, tails=DEFAULT_TAILS) -> list[dict]:
    """Every (precision, tail_queries) pair worth timing."""
    precisions = (0, 1) if screen_available else (0,)
    return [{"precision": p, "tail_queries": t}
            for p, t in itertools.product(precisions, tails)]


def _wall_timer(run) -> float:
    """Seconds of one synchronous call (bkd_query returns when done)."""
    t0 = time.perf_counter()
    run()
    return time.perf_counter() - t0


def autotune(tree, Q, k: int, screen_available: bool | None = None,
             tails=DEFAULT_TAILS, repeats: int = 2, timer=None,
             bkd=None) -> dict:
    """Times every candidate `repeats` times (best of), applies the fastest
    to `tree` and returns {"best": options, "timings": [(options, s)...]}
    sorted by time.  `screen_available`: whether the tree was built with
    precision=1 (None: probe by setting it).  `timer(run) -> seconds` and
    `bkd` (the binding module) can be replaced, e.g. in tests."""
    if bkd is None:
        import paper_1512_02831_gb300 as bkd
    timer = timer or _wall_timer
    if screen_available is None:
        try:
            bkd.bkd_set_option(tree, "precision", 1)
            screen_available = True
        except bkd.BkdError:
            screen_available = False
    timings = []
    for opts in candidates(screen_available, tails):
        for key, val in opts.items():
            bkd.bkd_set_option(tree, key, val)
        bkd.bkd_query(tree, Q, k)  # warm-up (workspace, caches)
        best = min(timer(lambda: bkd.bkd_query(tree, Q, k))
                   for _ in range(max(1, repeats)))
        timings.append((opts, best))
    timings.sort(key=lambda x: x[1])
    best_opts = timings[0][0]
    for key, val in best_opts.items():
        bkd.bkd_set_option(tree, key, val)
    return {"best": best_opts, "timings": timings}
