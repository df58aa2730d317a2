"""Parity bar between the CUDA path and the binary64 oracle.

For every query:
  * gap-exempt queries -- the oracle's k-th and (k+1)-th distances differ by
    less than 1e-6 relative -- may return any valid k-nearest set;
  * all other queries must return the oracle's index row exactly, order
    included;
  * every returned float32 distance is within 1e-5 relative (floor 1e-30) of
    the binary64 distance of the returned index;
  * every returned index is a valid neighbour: binary64 distance at most the
    oracle's k-th distance times (1 + 1e-5), no index repeated;
  * returned distances are non-decreasing along each row.
"""
from __future__ import annotations

import numpy as np

import oracle

REL_GAP = 1e-6
REL_DIST = 1e-5


def check(P, Q, k, idx, dist, ref, rows=None, exact_all=True):
    """Asserts the parity bar; ``rows`` selects which queries of Q the
    oracle result ``ref`` covers (default: all).  With ``exact_all`` the
    exempt queries must match the oracle exactly too (this implementation
    resolves near ties in binary64, so it can)."""
    idx = np.asarray(idx)
    dist = np.asarray(dist)
    if rows is None:
        rows = np.arange(Q.shape[0])
    rows = np.asarray(rows)
    gi, gd = idx[rows], dist[rows].astype(np.float64)
    m = len(rows)
    assert gi.shape == (m, k) and gd.shape == (m, k)
    exempt = ref.gap_exempt(REL_GAP)
    same = (gi == ref.idx).all(axis=1)
    bad = np.nonzero(~exempt & ~same)[0]
    assert bad.size == 0, (
        f"{bad.size} non-exempt queries differ from the oracle, e.g. query "
        f"{rows[bad[0]]}: gpu {gi[bad[0]].tolist()} oracle "
        f"{ref.idx[bad[0]].tolist()}")
    assert (gi >= 0).all() and (gi < P.shape[0]).all(), "index out of range"
    srt = np.sort(gi, axis=1)
    assert (np.diff(srt, axis=1) != 0).all(), "repeated index in a row"
    d64 = oracle.pair_dist(P, Q, np.repeat(rows, k), gi.ravel()).reshape(m, k)
    err = np.abs(gd - d64)
    lim = REL_DIST * np.maximum(d64, 1e-30)
    worst = np.argmax(err - lim)
    assert (err <= lim).all(), (
        f"distance off: query {rows[worst // k]} got {gd.flat[worst]} "
        f"binary64 {d64.flat[worst]}")
    assert (d64 <= ref.dist[:, -1:] * (1 + REL_DIST) + 1e-30).all(), \
        "returned a point farther than the k-th neighbour"
    assert (np.diff(gd, axis=1) >= 0).all(), "distances not non-decreasing"
    if exact_all:
        diff = np.nonzero(~same)[0]
        assert diff.size == 0, (
            f"{diff.size} exempt queries differ from the oracle, e.g. query "
            f"{rows[diff[0]]}: gpu {gi[diff[0]].tolist()} oracle "
            f"{ref.idx[diff[0]].tolist()}")
    return {"queries": m, "exempt": int(exempt.sum())}
