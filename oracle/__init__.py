"""Binary64 CPU oracle for exact k-nearest-neighbour search.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA path and never imports it.

Two implementations, both in ``bkd_oracle.c`` (plain C, OpenMP over queries):

* :func:`brute_knn` -- the definition of the problem in Sec. 2.2 of Gieseke et
  al. ("Bigger Buffer k-d Trees on Multi-Many-Core Systems"): score every
  reference point, keep the k+1 smallest keys (D, index).
* :func:`build_tree` / :func:`tree_knn` -- the classical k-d tree of
  Sec. 2.3 (median splits cycling through the dimensions, top-down descent,
  bottom-up backtracking with hyperplane pruning).

Distances are squared Euclidean distances formed in binary64 from the float32
inputs, terms added in dimension order.  Ties go to the smaller reference
index.  Each query also reports the (k+1)-th distance (``next``).

* :func:`outlier_scores` -- the proximity-based outlier score of Sec. 4.3 (a
  point's average Euclidean distance to its k nearest other points), from
  the brute-force definition above.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bkd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compiles ``bkd_oracle.c`` (or ``src``) into a shared library."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-shared", "-fPIC", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def bind(path: str):
    """Loads an oracle library from ``path`` and declares its signatures."""
    lib = ctypes.CDLL(path)
    lib.bkdo_brute.argtypes = [
        _f32p, ctypes.c_int64, ctypes.c_int, _f32p, ctypes.c_int64,
        ctypes.c_int, _i64p, _f64p, _f64p, ctypes.c_int]
    lib.bkdo_tree_build.argtypes = [
        _f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _f32p,
        _i64p, _f32p, _i64p, ctypes.c_int]
    lib.bkdo_tree_query.argtypes = [
        ctypes.c_int64, ctypes.c_int, ctypes.c_int, _f32p, _i64p,
        _f32p, _i64p, _f32p, ctypes.c_int64, ctypes.c_int, _i64p,
        _f64p, _f64p, _i64p, ctypes.c_int]
    lib.bkdo_pair_dist.argtypes = [
        _f32p, ctypes.c_int64, ctypes.c_int, _f32p, ctypes.c_int64,
        _i64p, _i64p, ctypes.c_int64, _f64p]
    lib.bkdo_max_threads.restype = ctypes.c_int
    for f in (lib.bkdo_brute, lib.bkdo_tree_build, lib.bkdo_tree_query,
              lib.bkdo_pair_dist):
        f.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.ndim != 2:
        raise ValueError("expected an (rows, d) array")
    return a


def max_threads() -> int:
    return int(_load().bkdo_max_threads())


class Result:
    """k nearest neighbours of m queries: ``idx`` (m, k) int64, ``dist``
    (m, k) float64 squared distances, ``next`` (m,) float64 (k+1)-th
    distance (+inf when k == n)."""

    def __init__(self, idx, dist, nxt, leaves=None):
        self.idx, self.dist, self.next, self.leaves = idx, dist, nxt, leaves

    def gap_exempt(self, rel: float = 1e-6) -> np.ndarray:
        """Queries whose k-th and (k+1)-th distances differ by less than
        ``rel`` relative: the k-th neighbour is not well defined there."""
        dk = self.dist[:, -1]
        return (self.next - dk) < rel * np.maximum(dk, 1e-30)


def brute_knn(P, Q, k: int, threads: int = 0, lib=None) -> Result:
    """Exact kNN by scoring every reference point (definition, Sec. 2.2)."""
    P, Q = _f32(P), _f32(Q)
    n, d = P.shape
    m = Q.shape[0]
    if Q.shape[1] != d:
        raise ValueError("P and Q differ in dimension")
    idx = np.empty((m, k), np.int64)
    dist = np.empty((m, k), np.float64)
    nxt = np.empty(m, np.float64)
    rc = _load(lib).bkdo_brute(_p(P, _f32p), n, d, _p(Q, _f32p), m, k,
                            _p(idx, _i64p), _p(dist, _f64p), _p(nxt, _f64p),
                            threads)
    if rc != 0:
        raise ValueError("oracle brute force rejected its arguments")
    return Result(idx, dist, nxt)


class Tree:
    """Classical k-d tree of height h (Sec. 2.3): ``split`` (2^h - 1,)
    float32 in heap order, ``perm`` (n,) original index of each leaf-structure
    position, ``pts`` (n, d) rearranged points, ``leaf_lo`` (2^h + 1,)
    leaf bounds."""

    def __init__(self, P, h: int, threads: int = 0, lib=None):
        self._lib = _load(lib)
        P = _f32(P)
        n, d = P.shape
        self.n, self.d, self.h = n, d, h
        self.split = np.empty(max((1 << h) - 1, 1), np.float32)
        self.perm = np.empty(n, np.int64)
        self.pts = np.empty((n, d), np.float32)
        self.leaf_lo = np.empty((1 << h) + 1, np.int64)
        rc = self._lib.bkdo_tree_build(
            _p(P, _f32p), n, d, h, _p(self.split, _f32p),
            _p(self.perm, _i64p), _p(self.pts, _f32p),
            _p(self.leaf_lo, _i64p), threads)
        if rc != 0:
            raise ValueError("oracle tree build rejected its arguments")

    def leaf_of_point(self) -> np.ndarray:
        """Leaf id of every original reference index."""
        sizes = np.diff(self.leaf_lo)
        leaf_at_pos = np.repeat(np.arange(1 << self.h), sizes)
        out = np.empty(self.n, np.int64)
        out[self.perm] = leaf_at_pos
        return out

    def knn(self, Q, k: int, threads: int = 0) -> Result:
        Q = _f32(Q)
        if Q.shape[1] != self.d:
            raise ValueError("query dimension differs from the tree's")
        m = Q.shape[0]
        idx = np.empty((m, k), np.int64)
        dist = np.empty((m, k), np.float64)
        nxt = np.empty(m, np.float64)
        leaves = np.empty(m, np.int64)
        rc = self._lib.bkdo_tree_query(
            self.n, self.d, self.h, _p(self.split, _f32p),
            _p(self.perm, _i64p), _p(self.pts, _f32p),
            _p(self.leaf_lo, _i64p), _p(Q, _f32p), m, k, _p(idx, _i64p),
            _p(dist, _f64p), _p(nxt, _f64p), _p(leaves, _i64p), threads)
        if rc != 0:
            raise ValueError("oracle tree query rejected its arguments")
        return Result(idx, dist, nxt, leaves)


def build_tree(P, h: int, threads: int = 0, lib=None) -> Tree:
    return Tree(P, h, threads, lib)


def tree_knn(P, Q, k: int, h: int, threads: int = 0, lib=None) -> Result:
    return Tree(P, h, threads, lib).knn(Q, k, threads)


def pair_dist(P, Q, qi, pi) -> np.ndarray:
    """binary64 squared distances D(Q[qi[j]], P[pi[j]])."""
    P, Q = _f32(P), _f32(Q)
    qi = np.ascontiguousarray(qi, np.int64).ravel()
    pi = np.ascontiguousarray(pi, np.int64).ravel()
    if qi.shape != pi.shape:
        raise ValueError("qi and pi differ in length")
    out = np.empty(qi.shape[0], np.float64)
    rc = _load().bkdo_pair_dist(_p(P, _f32p), P.shape[0], P.shape[1],
                                _p(Q, _f32p), Q.shape[0], _p(qi, _i64p),
                                _p(pi, _i64p), qi.shape[0], _p(out, _f64p))
    if rc != 0:
        raise ValueError("pair index out of range")
    return out


def outlier_scores(P, k: int, threads: int = 0) -> np.ndarray:
    """Outlier score of Sec. 4.3 (points ranked by the mean distance to
    their k nearest neighbours, queries = the reference set): for every
    point i, the mean of the binary64 Euclidean distances to
    its k nearest neighbours among the other points.  The neighbours are the
    first k+1 of the (distance, index) order of :func:`brute_knn` with the
    point's own index removed -- or, when k+1 exact duplicates of smaller
    index fill the row so that i is not in it, the last one removed."""
    P = _f32(P)
    n = P.shape[0]
    res = brute_knn(P, P, k + 1, threads)
    own = res.idx == np.arange(n)[:, None]
    drop = np.where(own.any(axis=1), own.argmax(axis=1), k)
    keep = np.ones(res.idx.shape, bool)
    keep[np.arange(n), drop] = False
    return np.sqrt(res.dist[keep].reshape(n, k)).mean(axis=1)
