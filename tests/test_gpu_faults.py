"""Failure paths reached from the host, without faulting the GPU.

bkd_test_fail_alloc makes the nth device or pinned host allocation of the
library fail as if the memory were exhausted.  Every call that meets such a
failure must return BKD_ENOMEM, and the library must stay usable: a failed
build leaves nothing behind, a failed query leaves its tree answering the
next query correctly, a failed server open leaves the tree serving."""
import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def hook_off():
    yield
    bkd.bkd_test_fail_alloc(0)


def _data():
    P = workloads.uniform(6000, 5, 1)
    Q = workloads.uniform(500, 5, 2)
    return P, Q, oracle.brute_knn(P, Q, 6)


@pytest.mark.parametrize("opts", [{}, {"precision": 1},
                                  {"precision": 1, "screen_kernel": 2},
                                  {"chunks": 3}])
def test_every_build_allocation_can_fail_cleanly(opts):
    P, Q, ref = _data()
    failed = 0
    for nth in range(1, 40):
        bkd.bkd_test_fail_alloc(nth)
        try:
            tree = bkd.bkd_build(P, 5, **opts)
        except bkd.BkdError as e:
            assert e.code == bkd.BKD_ENOMEM, e
            failed += 1
            continue
        finally:
            bkd.bkd_test_fail_alloc(0)
        # the build needed fewer than nth allocations: the query may meet it
        bkd.bkd_free(tree)
        break
    assert failed >= 5
    tree = bkd.bkd_build(P, 5, **opts)
    idx, dist = bkd.bkd_query(tree, Q, 6)
    bkd.bkd_free(tree)
    check(P, Q, 6, idx, dist, ref)


@pytest.mark.parametrize("precision,kernel", [(0, 0), (1, 0), (1, 1)])
def test_every_query_allocation_can_fail_and_the_tree_stays_usable(precision,
                                                                   kernel):
    P, Q, ref = _data()
    tree = bkd.bkd_build(P, 5, precision=1, screen_kernel=2)
    bkd.bkd_set_option(tree, "precision", precision)
    bkd.bkd_set_option(tree, "screen_kernel", kernel)
    try:
        failed = 0
        for nth in range(1, 30):
            # each round grows the workspace again: a larger query set
            Qn = np.concatenate([Q] * (nth + 1))
            bkd.bkd_test_fail_alloc(nth)
            try:
                bkd.bkd_query(tree, Qn, 6)
            except bkd.BkdError as e:
                assert e.code == bkd.BKD_ENOMEM, e
                failed += 1
            finally:
                bkd.bkd_test_fail_alloc(0)
            idx, dist = bkd.bkd_query(tree, Q, 6)
            check(P, Q, 6, idx, dist, ref)
        assert failed >= 5
    finally:
        bkd.bkd_free(tree)


def test_server_open_allocation_failure():
    P, Q, ref = _data()
    tree = bkd.bkd_build(P, 5)
    try:
        for nth in (1, 5, 12, 21):
            bkd.bkd_test_fail_alloc(nth)
            with pytest.raises(bkd.BkdError) as e:
                bkd.Server(tree, k_max=6, max_queries=1000)
            bkd.bkd_test_fail_alloc(0)
            assert e.value.code == bkd.BKD_ENOMEM
        srv = bkd.Server(tree, k_max=6, max_queries=1000)
        t = srv.submit(Q, 6)
        while srv.step():
            pass
        assert srv.status(t) == bkd.BKD_BATCH_DONE
        idx, dist = srv.result(t)
        srv.close()
        check(P, Q, 6, idx, dist, ref)
    finally:
        bkd.bkd_free(tree)


def test_fail_alloc_rejects_negative():
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_test_fail_alloc(-1)
    assert e.value.code == bkd.BKD_EINVAL
