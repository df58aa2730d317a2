"""Tall trees: heights 17, 18, 20 and 24 (the bigger-tree, d = 27 and
serving workloads use 18-20), with leaves of one to three points so that the
trees fit a test.  At these heights the traversal state's level mask, the
heap indices of the top tree (up to 2^25 - 2) and the per-node box array
(2^(h+1) - 1 boxes) reach sizes the other tests never touch.  Each case runs
the float32 path (and the BF16 screen where its data fits) against the
binary64 oracle on a sample of the queries."""
import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.mark.parametrize("h,n,d,screen", [
    (17, (1 << 18) + 3, 4, True),
    (18, (1 << 19) + 123, 3, True),
    (20, 1 << 21, 5, True),
    (24, (1 << 24) + 5, 2, False),
])
def test_tall_tree_matches_oracle(h, n, d, screen):
    params = workloads.mixture_params(d, 32, 0.02, 0.2, h)
    P = workloads.mixture(n, params, 1)
    Q = workloads.mixture(3000, params, 2)
    k = 10
    opts = {"precision": 1} if screen else {}
    tree = bkd.bkd_build(P, h, **opts)
    try:
        shape = bkd.bkd_tree_shape(tree)
        assert shape["height"] == h and not shape["chunked"]
        res = []
        for prec in ((0, 1) if screen else (0,)):
            for tail in (0, -1):
                bkd.bkd_set_option(tree, "precision", prec)
                bkd.bkd_set_option(tree, "tail_queries", tail)
                idx, dist = bkd.bkd_query(tree, Q, k)
                assert bkd.bkd_get_stat(tree, "rounds") > 0 or tail != 0
                res.append((idx, dist))
    finally:
        bkd.bkd_free(tree)
    for idx, dist in res[1:]:
        assert np.array_equal(idx, res[0][0])
        assert np.array_equal(dist, res[0][1])
    rows = np.arange(300)
    check(P, Q[rows], k, res[0][0][rows], res[0][1][rows],
          oracle.brute_knn(P, Q[rows], k))
