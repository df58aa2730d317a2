"""Pins for the binary64 oracle (CPU only).

The oracle is trusted for parity only because these tests tie it to things
other than itself:
  * hand-worked exact cases (tests/golden/hand_cases.json, Sec. 2.2 problem
    statement + the smaller-index tie rule);
  * a closed form: on the vertices of the unit hypercube {0,1}^d the squared
    distance between two vertices is their Hamming distance, so the exact
    neighbour order is (popcount(a xor b), b);
  * exact rational arithmetic (fractions.Fraction) on tiny random inputs: the
    binary64 distances must lie within the binary64 error bound of the exact
    value, and the order must match wherever the exact gap exceeds it;
  * the k-d tree's construction invariants (Sec. 2.3: median split in
    dimension level mod d, (almost) equal halves, contiguous leaves);
  * the k-d tree search (Sec. 2.3 backtracking) must equal brute force on
    every query, including data with many exact ties; height 0 reduces it to
    brute force itself;
  * mutation checks: plausible mistakes planted in a copy of the oracle source
    (wrong tie rule, strict pruning, dropped term, wrong sign, wrong median
    position) make at least one of the pins above fail.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def _num(v):
    return math.inf if v == "Infinity" else float(v)


def _hand_cases():
    with open(GOLDEN) as f:
        data = json.load(f)
    for case in data["cases"]:
        P = np.array(case["P"], np.float32)
        for qc in case["queries"]:
            yield case["name"], P, qc


def check_hand_cases(oracle, lib=None):
    """Returns a list of failure strings (empty when all hand cases hold)."""
    bad = []
    for name, P, qc in _hand_cases():
        Q = np.array([qc["q"]], np.float32)
        k = qc["k"]
        n = P.shape[0]
        results = [("brute", oracle.brute_knn(P, Q, k, lib=lib))]
        for h in range(0, int(math.log2(n)) + 1):
            results.append((f"tree h={h}",
                            oracle.tree_knn(P, Q, k, h, lib=lib)))
        for label, r in results:
            if list(r.idx[0]) != qc["idx"]:
                bad.append(f"{name} {qc['q']} {label}: idx {list(r.idx[0])}")
            if list(r.dist[0]) != [float(x) for x in qc["dist"]]:
                bad.append(f"{name} {qc['q']} {label}: dist {list(r.dist[0])}")
            if r.next[0] != _num(qc["next"]):
                bad.append(f"{name} {qc['q']} {label}: next {r.next[0]}")
    return bad


def hypercube(d):
    """Vertices of {0,1}^d; vertex i has coordinate j = bit j of i."""
    i = np.arange(1 << d)
    return ((i[:, None] >> np.arange(d)[None, :]) & 1).astype(np.float32)


def check_hypercube(oracle, lib=None):
    bad = []
    for d in (3, 5, 7):
        P = hypercube(d)
        n = P.shape[0]
        pop = np.array([bin(x).count("1") for x in range(n)])
        for k in (1, d + 1, n):
            for label, fn in (
                    ("brute", lambda: oracle.brute_knn(P, P, k, lib=lib)),
                    ("tree", lambda: oracle.tree_knn(P, P, k, min(d, 4),
                                                     lib=lib))):
                r = fn()
                for a in range(n):
                    ham = pop[a ^ np.arange(n)]
                    order = np.lexsort((np.arange(n), ham))
                    if not np.array_equal(r.idx[a], order[:k]):
                        bad.append(f"hypercube d={d} k={k} {label} a={a}")
                        break
                    if not np.array_equal(r.dist[a], ham[order[:k]]):
                        bad.append(f"hypercube dist d={d} k={k} {label}")
                        break
    return bad


def check_tree_vs_brute(oracle, lib=None, seeds=range(6)):
    """Tree search equals brute force, on tie-heavy integer data and on
    continuous data."""
    bad = []
    for seed in seeds:
        rng = np.random.default_rng(100 + seed)
        d = int(rng.integers(1, 6))
        n = int(rng.integers(8, 400))
        h = int(rng.integers(0, int(math.log2(n)) + 1))
        k = int(rng.integers(1, min(n, 12) + 1))
        for kind in ("grid", "cont"):
            if kind == "grid":
                P = rng.integers(0, 4, (n, d)).astype(np.float32)
                Q = rng.integers(-1, 5, (60, d)).astype(np.float32) * 0.5
            else:
                P = rng.standard_normal((n, d)).astype(np.float32)
                Q = rng.standard_normal((60, d)).astype(np.float32)
            rb = oracle.brute_knn(P, Q, k, lib=lib)
            rt = oracle.tree_knn(P, Q, k, h, lib=lib)
            if not (np.array_equal(rb.idx, rt.idx)
                    and np.array_equal(rb.dist, rt.dist)
                    and np.array_equal(rb.next, rt.next)):
                bad.append(f"tree!=brute seed={seed} {kind} n={n} d={d} "
                           f"h={h} k={k}")
    return bad


def check_tree_structure(oracle, P, h, lib=None):
    bad = []
    t = oracle.build_tree(P, h, lib=lib)
    n, d = P.shape
    sizes = np.diff(t.leaf_lo)
    if t.leaf_lo[0] != 0 or t.leaf_lo[-1] != n or np.any(sizes < 1):
        bad.append("leaves do not tile [0, n)")
    if sizes.max() - sizes.min() > 1:
        bad.append("leaf sizes differ by more than one")
    if not np.array_equal(np.sort(t.perm), np.arange(n)):
        bad.append("perm is not a permutation")
    if not np.array_equal(t.pts, P[t.perm]):
        bad.append("pts is not P permuted")

    def walk(node, level, lo, hi):
        if level == h:
            leaf = node - ((1 << h) - 1)
            if (t.leaf_lo[leaf], t.leaf_lo[leaf + 1]) != (lo, hi):
                bad.append(f"leaf {leaf} bounds")
            return
        s = level % d
        mid = lo + (hi - lo) // 2
        keys = list(zip(t.pts[lo:hi, s].tolist(), t.perm[lo:hi].tolist()))
        left, right = keys[:mid - lo], keys[mid - lo:]
        if left and max(left) > min(right):
            bad.append(f"node {node}: left/right keys not separated")
        if t.split[node] != t.pts[mid:hi, s].min():
            bad.append(f"node {node}: split is not the right half's "
                       "smallest value")
        walk(2 * node + 1, level + 1, lo, mid)
        walk(2 * node + 2, level + 1, mid, hi)

    walk(0, 0, 0, n)
    return bad


# ------------------------------------------------------------------- tests
def test_hand_cases(oracle_mod):
    assert check_hand_cases(oracle_mod) == []


def test_hypercube_closed_form(oracle_mod):
    assert check_hypercube(oracle_mod) == []


def test_line_closed_form(oracle_mod):
    """Points at the integers 0..n-1 on a line (in a scrambled index order);
    for a query at j + f with 0 < f < 1/2 the neighbours come in the order
    j, j+1, j-1, j+2, j-2, ... while both sides last."""
    n = 64
    rng = np.random.default_rng(5)
    order = rng.permutation(n)          # order[i] = position of index i
    P = order.astype(np.float32)[:, None]
    where = np.argsort(order)           # where[x] = index at position x
    j, f = 30, 0.25
    Q = np.array([[j + f]], np.float32)
    expect = [j]
    for s in range(1, 20):
        expect += [j + s, j - s]
    k = len(expect)
    for r in (oracle_mod.brute_knn(P, Q, k),
              oracle_mod.tree_knn(P, Q, k, 3)):
        assert list(r.idx[0]) == [int(where[x]) for x in expect]


def test_exact_rational_bound(oracle_mod):
    """binary64 distances against exact rationals (error bound (d+2)u,
    u = 2^-53); order identical wherever exact gaps exceed twice the bound."""
    rng = np.random.default_rng(11)
    for trial in range(12):
        d = int(rng.integers(1, 9))
        n = int(rng.integers(5, 40))
        P = (rng.standard_normal((n, d)) * rng.choice([1e-3, 1, 1e3])
             ).astype(np.float32)
        Q = (rng.standard_normal((4, d)) * 2).astype(np.float32)
        k = int(rng.integers(1, n + 1))
        r = oracle_mod.brute_knn(P, Q, k)
        gam = (d + 2) * 2.0 ** -53 * 1.01
        for qi in range(Q.shape[0]):
            exact = [sum((Fraction(float(Q[qi, j])) - Fraction(float(P[i, j])))
                         ** 2 for j in range(d)) for i in range(n)]
            rank = sorted(range(n), key=lambda i: (exact[i], i))
            for j in range(k):
                e = exact[r.idx[qi, j]]
                assert abs(Fraction(r.dist[qi, j]) - e) <= Fraction(gam) * e
            # positions whose exact neighbours are separated by > 2 gamma
            for j in range(k):
                a = exact[rank[j]]
                lo = exact[rank[j - 1]] if j > 0 else None
                hi = exact[rank[j + 1]] if j + 1 < n else None
                sep = all(b is None or abs(b - a) > 2 * Fraction(gam) * a
                          for b in (lo, hi))
                if sep:
                    assert r.idx[qi, j] == rank[j]


@pytest.mark.parametrize("n,d,h", [(1000, 3, 5), (777, 10, 6), (64, 2, 6),
                                   (4096, 10, 8), (33, 1, 2)])
def test_tree_structure(oracle_mod, n, d, h):
    P = workloads.uniform(n, d, n + d)
    assert check_tree_structure(oracle_mod, P, h) == []


def test_tree_structure_with_duplicate_coordinates(oracle_mod):
    rng = np.random.default_rng(3)
    P = rng.integers(0, 3, (500, 4)).astype(np.float32)
    assert check_tree_structure(oracle_mod, P, 5) == []


def test_tree_equals_brute_small(oracle_mod):
    assert check_tree_vs_brute(oracle_mod, seeds=range(40)) == []


@pytest.mark.parametrize("kind", ["uniform", "mixture"])
def test_tree_equals_brute_exhaustive_4096(oracle_mod, kind):
    """All n <= 4096 sizes swept coarsely, every query checked."""
    rng = np.random.default_rng(9)
    params = workloads.mixture_params(10, 32, 0.02, 0.2, 0)
    for n in (17, 256, 1000, 4096):
        d = 10
        if kind == "uniform":
            P = workloads.uniform(n, d, 1)
            Q = workloads.uniform(300, d, 2)
        else:
            P = workloads.mixture(n, params, 1)
            Q = workloads.mixture(300, params, 2)
        for h in sorted({0, 2, int(math.log2(n)) // 2,
                         int(math.log2(n))}):
            k = int(rng.integers(1, min(n, 20) + 1))
            rb = oracle_mod.brute_knn(P, Q, k)
            rt = oracle_mod.tree_knn(P, Q, k, h)
            assert np.array_equal(rb.idx, rt.idx)
            assert np.array_equal(rb.dist, rt.dist)
            assert np.array_equal(rb.next, rt.next)


def test_tree_prunes(oracle_mod):
    """Backtracking with hyperplane pruning (Sec. 2.3) visits far fewer than
    all leaves on low-dimensional data."""
    P = workloads.uniform(1 << 14, 3, 0)
    Q = workloads.uniform(500, 3, 1)
    r = oracle_mod.tree_knn(P, Q, 5, 8)
    assert r.leaves.max() <= 256
    assert r.leaves.mean() < 16


def test_rows_ascending_and_valid(oracle_mod):
    P = workloads.uniform(3000, 6, 4)
    Q = workloads.uniform(200, 6, 5)
    r = oracle_mod.tree_knn(P, Q, 15, 7)
    key_ok = (np.diff(r.dist, axis=1) > 0) | (
        (np.diff(r.dist, axis=1) == 0) & (np.diff(r.idx, axis=1) > 0))
    assert key_ok.all()
    assert (r.next >= r.dist[:, -1]).all()
    qi = np.repeat(np.arange(200), 15)
    assert np.array_equal(oracle_mod.pair_dist(P, Q, qi, r.idx.ravel()),
                          r.dist.ravel())


def test_rejects_bad_arguments(oracle_mod):
    P = workloads.uniform(16, 2, 0)
    with pytest.raises(ValueError):
        oracle_mod.brute_knn(P, P, 17)
    with pytest.raises(ValueError):
        oracle_mod.build_tree(P, 5)       # 2^5 leaves > 16 points
    with pytest.raises(ValueError):
        oracle_mod.brute_knn(P, P, 0)


# ---------------------------------------------------------------- mutants
MUTANTS = {
    "tie rule flipped": ("return da < db || (da == db && ia < ib);",
                         "return da < db || (da == db && ia > ib);"),
    "strict pruning": ("if (plane <= bound)", "if (plane < bound)"),
    "last term dropped": ("for (int j = 0; j < d; ++j) {\n    double t",
                          "for (int j = 0; j < d - 1; ++j) {\n    double t"),
    "wrong sign": ("double t = (double)q[j] - (double)x[j];",
                   "double t = (double)q[j] + (double)x[j];"),
    "median one off": ("int64_t mid = lo + (hi - lo) / 2;",
                       "int64_t mid = lo + (hi - lo + 1) / 2;"),
    "descent flipped": ("int64_t near_child = q[s] < sv ?",
                        "int64_t near_child = q[s] >= sv ?"),
    "prune on k-th not (k+1)-th": (
        "double bound = *cnt < K ? INFINITY : L[K - 1].dist;",
        "double bound = *cnt < K - 1 ? INFINITY : L[K - 2].dist;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(oracle_mod, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle_mod._SRC).read()
    assert src.count(old) == 1, name
    mpath = tmp_path / "mut.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle_mod.bind(oracle_mod.build(force=True, src=str(mpath),
                                           out=str(tmp_path / "mut.so")))
    failures = check_hand_cases(oracle_mod, lib)
    failures += check_hypercube(oracle_mod, lib)
    failures += check_tree_vs_brute(oracle_mod, lib, seeds=range(40))
    failures += check_tree_structure(oracle_mod,
                                     workloads.uniform(200, 3, 1), 4, lib)
    assert failures, f"mutant '{name}' passed every pin"


def test_outlier_scores_hand_cases(oracle_mod):
    """Sec. 4.3 outlier score against hand-computed values (own index
    removed from the k+1 list, or the last entry when duplicates fill it)."""
    data = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                       "outlier_cases.json")))
    for case in data["cases"]:
        P = np.array(case["P"], np.float32)
        got = oracle_mod.outlier_scores(P, case["k"])
        assert np.allclose(got, case["score"], rtol=0, atol=1e-12), \
            (case["name"], got)


def test_outlier_scores_grid_closed_form(oracle_mod):
    """Closed forms on the integer grid {0..9}^2: every point has at least
    two neighbours at distance 1, so k = 2 scores 1 everywhere; with k = 4
    an interior point has four at 1 (score 1), a corner two at 1, one at
    sqrt 2 and then two at 2 (score (1 + 1 + sqrt 2 + 2) / 4), and an edge
    point three at 1 and then two at sqrt 2 (score (3 + sqrt 2) / 4)."""
    g = np.stack(np.meshgrid(np.arange(10), np.arange(10), indexing="ij"),
                 -1).reshape(-1, 2).astype(np.float32)
    s2 = oracle_mod.outlier_scores(g, 2)
    assert np.allclose(s2, 1.0)
    s4 = oracle_mod.outlier_scores(g, 4)
    inside = (g[:, 0] > 0) & (g[:, 0] < 9) & (g[:, 1] > 0) & (g[:, 1] < 9)
    assert np.allclose(s4[inside], 1.0)
    corner = ((g[:, 0] == 0) | (g[:, 0] == 9)) & ((g[:, 1] == 0)
                                                  | (g[:, 1] == 9))
    assert np.allclose(s4[corner], (1 + 1 + np.sqrt(2) + 2) / 4)
    edge = ~inside & ~corner
    assert np.allclose(s4[edge], (3 + np.sqrt(2)) / 4)
