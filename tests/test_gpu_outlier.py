"""The outlier score of Sec. 4.3 on the GPU (bkd_outlier_scores) against the
binary64 oracle: every reference point's mean Euclidean distance to its k
nearest other points, within the distance tolerance (1e-5 relative, the
square root halves the squared-distance error)."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads

pytestmark = pytest.mark.gpu

REL = 1e-5


def _check(got, ref):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref) / np.maximum(ref, 1e-30)
    worst = int(np.argmax(err))
    assert (err <= REL).all() or (np.abs(got - ref) <= 1e-30).all(), (
        f"point {worst}: gpu {got[worst]} oracle {ref[worst]}")


def test_outlier_hand_cases():
    data = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "outlier_cases.json")))
    for case in data["cases"]:
        P = np.array(case["P"], np.float32)
        tree = bkd.bkd_build(P, 1)
        try:
            got = bkd.bkd_outlier_scores(tree, case["k"])
        finally:
            bkd.bkd_free(tree)
        assert np.array_equal(got, np.array(case["score"], np.float32)), \
            (case["name"], got)


@pytest.mark.parametrize("opts", [{}, {"precision": 1}, {"chunks": 3},
                                  {"max_active": 3000}])
def test_outlier_scores_match_oracle(opts):
    params = workloads.mixture_params(5, 16, 0.02, 0.2, 0)
    P = workloads.with_duplicates(workloads.mixture(20000, params, 1), 0.01,
                                  4)
    k = 10
    ref = oracle.outlier_scores(P, k)
    tree = bkd.bkd_build(P, 6, **opts)
    try:
        got = bkd.bkd_outlier_scores(tree, k)
        assert bkd.bkd_get_stat(tree, "kernel_launches") > 0
    finally:
        bkd.bkd_free(tree)
    _check(got, ref)


def test_outlier_scores_device_output_and_errors():
    torch = pytest.importorskip("torch")
    P = workloads.uniform(5000, 3, 2)
    tree = bkd.bkd_build(P, 5)
    try:
        out = bkd.bkd_outlier_scores(tree, 7, device="cuda:0")
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), oracle.outlier_scores(P, 7))
        with pytest.raises(bkd.BkdError) as e:
            bkd.bkd_outlier_scores(tree, 0)
        assert e.value.code == bkd.BKD_EINVAL
        with pytest.raises(bkd.BkdError) as e:
            bkd.bkd_outlier_scores(tree, bkd.BKD_MAX_K)
        assert e.value.code == bkd.BKD_EUNSUPPORTED
    finally:
        bkd.bkd_free(tree)
