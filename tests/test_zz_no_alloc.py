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

import paper_1512_02831_gb300 as bkd
import workloads

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
    finally:
        bkd.bkd_free(tree)


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
