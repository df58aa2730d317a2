"""Continuous batching (bkd_serve_*): batches of uneven size and k, arriving
while others are in flight, share the LazySearch rounds; each batch's result
is the same alone and in the mix."""
import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = pytest.mark.gpu


def _serve(srv, arrivals, max_steps=200000):
    """arrivals: list of (step, submit-callable); returns tickets by index."""
    tickets = {}
    step = 0
    last = max(a for a, _ in arrivals)
    while True:
        for j, (a, submit) in enumerate(arrivals):
            if a == step:
                tickets[j] = submit()
        pending = srv.step()
        step += 1
        if step > last and pending == 0:
            return tickets
        assert step < max_steps


@pytest.mark.parametrize("precision,kernel", [(0, 0), (1, 0), (1, 1)])
def test_each_batch_same_alone_and_in_the_mix(precision, kernel):
    import torch
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 16, 6000, 8)
    P, Qall = w.points(), w.queries()
    opts = {"screen_kernel": kernel} if precision else {}
    tree = bkd.bkd_build(P, w.height, precision=precision, **opts)
    # (first query, batch size, k, arrival step, device buffers)
    spec = [(0, 1, 10, 0, False), (1, 37, 1, 0, True), (38, 500, 50, 1, False),
            (538, 1200, 10, 3, True), (1738, 3, 50, 3, False),
            (1741, 2000, 7, 5, False), (3741, 900, 25, 9, True),
            (4641, 1359, 50, 9, False)]
    try:
        alone = [bkd.bkd_query(tree, np.ascontiguousarray(Qall[a:a + m]), k)
                 for a, m, k, _, _ in spec]
        # fewer slots than queries in flight: later batches wait for slots
        srv = bkd.Server(tree, k_max=50, max_queries=2500)

        def submitter(a, m, k, dev):
            def go():
                Q = np.ascontiguousarray(Qall[a:a + m])
                return srv.submit(torch.from_numpy(Q).cuda() if dev else Q, k)
            return go

        tickets = _serve(srv, [(s[3], submitter(*s[:3], s[4])) for s in spec])
        for j, (a, m, k, _, dev) in enumerate(spec):
            assert srv.status(tickets[j]) == bkd.BKD_BATCH_DONE
            idx, dist = srv.result(tickets[j])
            if dev:
                idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
            assert np.array_equal(idx, alone[j][0]), j
            assert np.array_equal(dist, alone[j][1]), j
        a, m, k = spec[5][:3]
        check(P, Qall[a:a + m], k, alone[5][0], alone[5][1],
              oracle.brute_knn(P, Qall[a:a + m], k))
        srv.close()
    finally:
        bkd.bkd_free(tree)


@pytest.mark.parametrize("rescue,defer", [(1, 0), (3, 0), (384, 8),
                                          (3, 64)])
def test_rescued_and_deferred_queries_give_the_same_results(rescue, defer):
    """Batches older than `rescue` rounds have their remaining queries
    finished by the tail kernel, and with the buffer trigger (`defer`) a
    leaf holding fewer queries waits up to 4 rounds; every batch's result
    still equals a bkd_query of it alone (float32 and the warp screen)."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 16, 4000, 8)
    P, Qall = w.points(), w.queries()
    tree = bkd.bkd_build(P, w.height, precision=1, rescue_rounds=rescue,
                         defer_queries=defer)
    spec = [(0, 700, 10, 0), (700, 1300, 50, 1), (2000, 5, 1, 2),
            (2005, 1995, 10, 4)]
    try:
        for prec in (0, 1):
            bkd.bkd_set_option(tree, "precision", prec)
            alone = [bkd.bkd_query(tree, np.ascontiguousarray(Qall[a:a + m]),
                                   k) for a, m, k, _ in spec]
            srv = bkd.Server(tree, k_max=50, max_queries=4000)

            def submitter(a, m, k):
                return lambda: srv.submit(np.ascontiguousarray(Qall[a:a + m]),
                                          k)
            tickets = _serve(srv, [(s[3], submitter(*s[:3])) for s in spec])
            for j in range(len(spec)):
                assert srv.status(tickets[j]) == bkd.BKD_BATCH_DONE
                idx, dist = srv.result(tickets[j])
                assert np.array_equal(idx, alone[j][0]), (prec, j)
                assert np.array_equal(dist, alone[j][1]), (prec, j)
            srv.close()
        # switching the trigger off with flags still set: the next rounds
        # clear them and every batch still completes
        if defer:
            srv = bkd.Server(tree, k_max=50, max_queries=4000)
            a, m, k, _ = spec[3]
            t1 = srv.submit(np.ascontiguousarray(Qall[a:a + m]), k)
            for _ in range(3):
                srv.step()
            bkd.bkd_set_option(tree, "defer_queries", 0)
            steps = 0
            while srv.step():
                steps += 1
                assert steps < 100000
            assert srv.status(t1) == bkd.BKD_BATCH_DONE
            idx, dist = srv.result(t1)
            assert np.array_equal(idx, alone[3][0])
            srv.close()
    finally:
        bkd.bkd_free(tree)


def test_bad_batches_fail_alone():
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 14, 500, 6)
    P, Q = w.points(), w.queries()
    tree = bkd.bkd_build(P, w.height)
    try:
        srv = bkd.Server(tree, k_max=10, max_queries=400)
        with pytest.raises(bkd.BkdError):
            srv.submit(Q[:401].copy(), 5)        # more than the slots
        with pytest.raises(bkd.BkdError):
            srv.submit(Q[:10].copy(), 11)        # k above k_max
        bad = Q[:50].copy()
        bad[7, 2] = np.nan
        t_bad = srv.submit(bad, 5)
        t_good = srv.submit(Q[50:300].copy(), 5)
        t_empty = srv.submit(np.zeros((0, w.d), np.float32), 5)
        while srv.step():
            pass
        assert srv.status(t_bad) == bkd.BKD_EINVAL
        assert srv.status(t_good) == bkd.BKD_BATCH_DONE
        assert srv.status(t_empty) == bkd.BKD_BATCH_DONE
        idx, dist = srv.result(t_good)
        ref_i, ref_d = bkd.bkd_query(tree, Q[50:300].copy(), 5)
        assert np.array_equal(idx, ref_i) and np.array_equal(dist, ref_d)
        with pytest.raises(bkd.BkdError):
            srv.status(t_good)                   # terminal status read once
        srv.close()
    finally:
        bkd.bkd_free(tree)
