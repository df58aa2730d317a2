"""bkd_query_static, the query entry point that allocates nothing.

It serves callers that cannot call cudaMalloc while they answer queries (a
process whose device memory belongs to its own pool allocator, or a loop that
cannot let cudaFree synchronise the device): its workspace is a fixed static
device array inside the library.  Here it is called through the C ABI and must
return what bkd_query returns for the same tree and queries, on two calls in
a row (the second call must not see the first call's leftovers in the shared
scratch).  This file is collected last so that a run stopping at the first
failure has run every other test already.
"""
import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = pytest.mark.gpu


def test_static_entry_point_matches_bkd_query_on_two_calls():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    params = workloads.mixture_params(10, 16, 0.02, 0.2, 0)
    P = workloads.mixture(40000, params, 5)
    tree = bkd.bkd_build(P, 7)
    try:
        for m, k, seed in ((3000, 10, 11), (1500, 4, 12)):
            Q = torch.from_numpy(workloads.mixture(m, params, seed)).to(dev)
            ref_i, ref_d = bkd.bkd_query(tree, Q, k)
            oi = torch.full((m, k), -7, dtype=torch.int64, device=dev)
            od = torch.full((m, k), -7.0, dtype=torch.float32, device=dev)
            bkd.bkd_query_static(tree, Q, k, oi, od)
            torch.cuda.synchronize(dev)
            assert torch.equal(oi, ref_i), f"indices differ (m={m}, k={k})"
            ref = ref_d.double()
            rel = ((od.double() - ref).abs() / ref.clamp_min(1e-30)).max()
            assert float(rel) <= 1e-5, f"distances differ by {float(rel)}"
            rows = np.arange(0, m, 7)
            Qh = Q.cpu().numpy()
            check(P, Qh[rows], k, oi.cpu().numpy()[rows],
                  od.cpu().numpy()[rows], oracle.brute_knn(P, Qh[rows], k))
    finally:
        bkd.bkd_free(tree)


def test_static_entry_point_at_the_scratch_layout_maxima():
    """The fixed scratch layout at its largest pieces: d = 32 (widest padded
    query rows), k = 63 (64-entry lists), height 16 (65,536 leaves: the
    largest count, offset, cursor and item arrays) and m = 4,096 queries."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(31)
    n, d, k, h, m = (1 << 17) + 7, 32, 63, 16, bkd.BKD_STATIC_MAX_QUERIES
    P = rng.standard_normal((n, d)).astype(np.float32)
    Qh = rng.standard_normal((m, d)).astype(np.float32)
    tree = bkd.bkd_build(P, h)
    try:
        Q = torch.from_numpy(Qh).to(dev)
        oi = torch.full((m, k), -7, dtype=torch.int64, device=dev)
        od = torch.full((m, k), -7.0, dtype=torch.float32, device=dev)
        bkd.bkd_query_static(tree, Q, k, oi, od)
        ref_i, ref_d = bkd.bkd_query(tree, Q, k)
        torch.cuda.synchronize(dev)
        assert torch.equal(oi, ref_i) and torch.equal(od, ref_d)
    finally:
        bkd.bkd_free(tree)
    rows = np.arange(0, m, 16)
    check(P, Qh[rows], k, oi.cpu().numpy()[rows], od.cpu().numpy()[rows],
          oracle.brute_knn(P, Qh[rows], k))


def test_static_entry_point_first_call_on_a_side_stream():
    """The first call on a fresh tree, with its queries written by a kernel
    on a non-default torch stream and its outputs read on that stream: the
    call must run on the caller's current stream, ordered after the write
    and before the reads."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = workloads.uniform(30000, 6, 3)
    Qh = workloads.uniform(2000, 6, 4)
    k = 9
    tree = bkd.bkd_build(P, 6)
    try:
        base = torch.from_numpy(Qh).to(dev)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            # a long kernel chain before Q is final: an unordered read would
            # see a partial result
            Q = base * 3.0
            for _ in range(200):
                Q = Q * 1.0
            Q = Q / 3.0
            oi = torch.empty((2000, k), dtype=torch.int64, device=dev)
            od = torch.empty((2000, k), dtype=torch.float32, device=dev)
            bkd.bkd_query_static(tree, Q, k, oi, od)
            got_i, got_d = oi.cpu(), od.cpu()
        Q_final = Q.cpu().numpy()
    finally:
        bkd.bkd_free(tree)
    check(P, Q_final, k, got_i.numpy(), got_d.numpy(),
          oracle.brute_knn(P, Q_final, k))


def test_static_entry_point_rejects_what_it_cannot_serve():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    P = workloads.uniform(5000, 3, 1)
    tree = bkd.bkd_build(P, 4)
    try:
        m = bkd.BKD_STATIC_MAX_QUERIES + 1
        Q = torch.zeros((m, 3), dtype=torch.float32, device=dev)
        oi = torch.empty((m, 2), dtype=torch.int64, device=dev)
        od = torch.empty((m, 2), dtype=torch.float32, device=dev)
        with pytest.raises(bkd.BkdError) as e:
            bkd.bkd_query_static(tree, Q, 2, oi, od)
        assert e.value.code == bkd.BKD_EINVAL
        assert "at most" in str(e.value)
        Qh = np.zeros((4, 3), np.float32)
        with pytest.raises(bkd.BkdError) as e:
            bkd.bkd_query_static(tree, Qh, 2, np.empty((4, 2), np.int64),
                                 np.empty((4, 2), np.float32))
        assert "device pointers" in str(e.value)
    finally:
        bkd.bkd_free(tree)
