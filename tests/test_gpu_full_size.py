"""Parity at the bench's full size and launch configuration: the 2^26-point,
2^24-query mixture, BF16 screen on, default options (tail kernel automatic),
one bkd_query over all queries; a seeded sample of rows checked against the
oracle's k-d tree (binary64), element by element."""
import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_full_size_mixture_sampled_rows():
    import torch
    w = workloads.MIXTURE_64M
    P, Q = w.points(), w.queries()
    rows = np.sort(np.random.default_rng(5).choice(Q.shape[0], 2000,
                                                   replace=False))
    tree = bkd.bkd_build(P, w.height, precision=1)
    try:
        Qd = torch.from_numpy(Q).cuda()
        idx, dist = bkd.bkd_query(tree, Qd, w.k)
        sel = torch.from_numpy(rows).cuda()
        gi, gd = idx[sel].cpu().numpy(), dist[sel].cpu().numpy()
        assert bkd.bkd_get_stat(tree, "screen_pairs") > 0
    finally:
        bkd.bkd_free(tree)
    ref = oracle.build_tree(P, w.height).knn(Q[rows], w.k)
    check(P, Q[rows], w.k, gi, gd, ref)
