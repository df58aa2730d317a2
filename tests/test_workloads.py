"""The seeded input generators (no method arithmetic): determinism, the
stated distributions, and independence from the worker-thread count."""
import numpy as np

import workloads


def test_uniform_is_seeded_float32_in_unit_cube():
    a = workloads.uniform(5000, 7, 3)
    b = workloads.uniform(5000, 7, 3)
    assert a.dtype == np.float32 and a.shape == (5000, 7)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, workloads.uniform(5000, 7, 4))
    assert a.min() >= 0.0 and a.max() < 1.0
    assert abs(a.mean() - 0.5) < 0.01


def test_mixture_parameters():
    p = workloads.mixture_params(10, 32, 0.02, 0.2, 0)
    assert p.centers.shape == (32, 10)
    assert (p.centers >= 0).all() and (p.centers < 1).all()
    assert (p.sigmas >= 0.02).all() and (p.sigmas <= 0.2).all()
    assert abs(p.weights.sum() - 1.0) < 1e-12 and (p.weights > 0).all()


def test_mixture_mean_and_spread():
    p = workloads.mixture_params(4, 3, 0.05, 0.05, 1)
    x = workloads.mixture(200000, p, 2).astype(np.float64)
    # mean = sum_c w_c c_c; per-dimension variance = sum_c w_c (sigma^2 +
    # c_c^2) - mean^2 (a mixture of isotropic Gaussians)
    mean = p.weights @ p.centers
    var = p.weights @ (p.sigmas[:, None] ** 2 + p.centers ** 2) - mean ** 2
    assert np.allclose(x.mean(0), mean, atol=5e-3)
    assert np.allclose(x.var(0), var, rtol=0.03)


def test_mixture_independent_of_worker_threads(monkeypatch):
    p = workloads.mixture_params(3, 5, 0.02, 0.2, 0)
    n = 2 * workloads.BLOCK + 17
    monkeypatch.setattr(workloads, "_workers", lambda: 1)
    a = workloads.mixture(n, p, 9)
    monkeypatch.setattr(workloads, "_workers", lambda: 7)
    b = workloads.mixture(n, p, 9)
    assert np.array_equal(a, b)
    # block b of the draw depends on the seed and b only
    assert np.array_equal(a[:workloads.BLOCK],
                          workloads.mixture(workloads.BLOCK, p, 9))


def test_with_duplicates_copies_other_rows():
    P = workloads.uniform(10000, 5, 1)
    D = workloads.with_duplicates(P, 0.01, 2)
    assert D.shape == P.shape and D.dtype == np.float32
    changed = (D != P).any(1)
    assert changed.sum() <= 100
    # every changed row is an exact copy of an original row
    orig = {r.tobytes() for r in P}
    assert all(D[i].tobytes() in orig for i in np.flatnonzero(changed))
    _, counts = np.unique(D, axis=0, return_counts=True)
    assert (counts > 1).sum() >= 90      # ~100 rows now appear twice
    assert np.array_equal(workloads.with_duplicates(P, 0.0, 2), P)


def test_query_streams_are_independent_and_seeded():
    w = workloads.scaled(workloads.MIXTURE_64M, 4096, 500, 4)
    q0, q0b, q1 = w.queries(), w.queries(), w.queries(stream=1)
    assert np.array_equal(q0, q0b)
    assert not (q0[:, None, :] == q1[None, :, :]).all(-1).any()
    assert q0.shape == (500, 10)


def test_d27_workload_has_duplicates():
    w = workloads.scaled(workloads.MIXTURE_D27, 20000, 10, 6)
    P = w.points()
    assert P.shape == (20000, 27)
    _, counts = np.unique(P, axis=0, return_counts=True)
    assert (counts > 1).sum() >= 150     # 1% of the rows are copies
