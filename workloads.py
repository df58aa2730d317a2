"""Seeded synthetic inputs for the buffer k-d tree kNN path.

This module only draws random numbers: it holds none of the method's
arithmetic, and both the CUDA path's tests and the oracle read the arrays it
returns.  The paper's astronomy catalogues (photometric magnitudes and
light-curve features, Sec. 4.1) are not available, so the shapes and value
distributions below stand in for them:

* ``uniform``      -- i.i.d. uniform on [0, 1)^d (numpy PCG64, float32).
* ``mixture``      -- isotropic Gaussian mixture mimicking photometric colour
  features: component centres uniform in [0, 1]^d, widths log-uniform in
  [sigma_lo, sigma_hi], weights Dirichlet(1, ..., 1); a point picks a
  component by weight and adds sigma * N(0, I_d); it is not clipped.
* ``with_duplicates`` -- overwrites a seeded fraction of rows with exact
  copies of other rows (forces exact distance ties).

Large draws are split into fixed blocks of 2^20 rows, each block with its own
child of ``numpy.random.SeedSequence(seed)``, so the result is the same for
any number of worker threads.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

BLOCK = 1 << 20


def uniform(n: int, d: int, seed: int) -> np.ndarray:
    """(n, d) float32, i.i.d. uniform on [0, 1)."""
    return np.random.default_rng(seed).random((n, d), dtype=np.float32)


@dataclass(frozen=True)
class MixtureParams:
    centers: np.ndarray   # (c, d) float64
    sigmas: np.ndarray    # (c,) float64
    weights: np.ndarray   # (c,) float64


def mixture_params(d: int, components: int, sigma_lo: float, sigma_hi: float,
                   seed: int) -> MixtureParams:
    rng = np.random.default_rng(seed)
    centers = rng.random((components, d))
    sigmas = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi),
                                components))
    weights = rng.dirichlet(np.ones(components))
    return MixtureParams(centers, sigmas, weights)


def _workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def mixture(n: int, params: MixtureParams, seed: int) -> np.ndarray:
    """(n, d) float32 drawn from the Gaussian mixture ``params``."""
    d = params.centers.shape[1]
    out = np.empty((n, d), np.float32)
    nblocks = (n + BLOCK - 1) // BLOCK
    children = np.random.SeedSequence(seed).spawn(max(nblocks, 1))
    cdf = np.cumsum(params.weights)
    cdf /= cdf[-1]
    centers32 = params.centers.astype(np.float32)
    sigmas32 = params.sigmas.astype(np.float32)

    def fill(b: int) -> None:
        lo, hi = b * BLOCK, min(n, (b + 1) * BLOCK)
        rng = np.random.default_rng(children[b])
        comp = np.searchsorted(cdf, rng.random(hi - lo), side="right")
        comp = np.minimum(comp, len(cdf) - 1)
        z = rng.standard_normal((hi - lo, d), dtype=np.float32)
        z *= sigmas32[comp, None]
        z += centers32[comp]
        out[lo:hi] = z

    if nblocks <= 1:
        for b in range(nblocks):
            fill(b)
    else:
        with ThreadPoolExecutor(_workers()) as ex:
            list(ex.map(fill, range(nblocks)))
    return out


def with_duplicates(P: np.ndarray, fraction: float, seed: int) -> np.ndarray:
    """Copy of P in which round(fraction * n) seeded rows are overwritten by
    exact copies of other seeded rows."""
    P = np.array(P, dtype=np.float32, copy=True)
    n = P.shape[0]
    cnt = int(round(fraction * n))
    if cnt == 0 or n < 2:
        return P
    rng = np.random.default_rng(seed)
    dst = rng.choice(n, size=cnt, replace=False)
    src = rng.integers(0, n, size=cnt)
    P[dst] = P[src]
    return P


# ---------------------------------------------------------------- workloads
@dataclass(frozen=True)
class Workload:
    """One named kNN workload: reference set, query set, k and tree height."""
    name: str
    n: int
    m: int
    d: int
    k: int
    height: int
    kind: str               # "uniform" or "mixture"
    components: int = 32
    sigma_lo: float = 0.02
    sigma_hi: float = 0.2
    duplicates: float = 0.0

    def points(self) -> np.ndarray:
        if self.kind == "uniform":
            return uniform(self.n, self.d, 0)
        P = mixture(self.n, self._params(), 1)
        if self.duplicates:
            P = with_duplicates(P, self.duplicates, 3)
        return P

    def queries(self, m: int | None = None, stream: int = 0) -> np.ndarray:
        """Query set; ``stream`` > 0 draws an independent set of the same
        distribution (one per process when the queries are sharded)."""
        m = self.m if m is None else m
        if self.kind == "uniform":
            return uniform(m, self.d, 1 + 1000 * stream)
        return mixture(m, self._params(), 2 + 1000 * stream)

    def _params(self) -> MixtureParams:
        return mixture_params(self.d, self.components, self.sigma_lo,
                              self.sigma_hi, 0)

    def describe(self) -> dict:
        return {"workload": self.name, "n": self.n, "m": self.m, "d": self.d,
                "k": self.k, "height": self.height, "data": self.kind}


UNIFORM_64K = Workload("uniform n=65536 m=16384 d=10 k=10 h=8", 65536, 16384,
                       10, 10, 8, "uniform")
MIXTURE_64M = Workload("mixture32 n=2^26 m=2^24 d=10 k=10 h=16", 1 << 26,
                       1 << 24, 10, 10, 16, "mixture")
# the serving workload: the bench distribution at n = 2^30 (h = 20, leaves
# of 1,024 points, 43 GB of points), a pool of 2^24 queries that serving
# batches are sliced from
MIXTURE_1G = Workload("mixture32 n=2^30 m=2^24 d=10 k=10 h=20", 1 << 30,
                      1 << 24, 10, 10, 20, "mixture")
MIXTURE_D27 = Workload("mixture64+1%dup n=2^28 m=2^25 d=27 k=50 h=18", 1 << 28,
                       1 << 25, 27, 50, 18, "mixture", components=64,
                       sigma_lo=0.01, sigma_hi=0.3, duplicates=0.01)


def scaled(w: Workload, n: int, m: int, height: int) -> Workload:
    """Same distribution as ``w`` at a smaller size."""
    return Workload(f"{w.name} scaled n={n} m={m} h={height}", n, m, w.d, w.k,
                    height, w.kind, w.components, w.sigma_lo, w.sigma_hi,
                    w.duplicates)
