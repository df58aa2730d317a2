"""Parity of the CUDA path against the binary64 oracle (needs a GPU).

Sizes span several leaves, several query tiles of the leaf kernel and ragged
tails (n not a multiple of 2^h or of 4, m not a multiple of the tile).  Edge
cases: height 0 (one leaf = brute force), k = n, a single point, all points
identical, exact ties on integer grids, duplicate rows, queries equal to
reference points, far-away queries, every compiled dimension.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_cases.json")


def run(P, Q, k, h, **opts):
    """Build + query.  Unless a test says otherwise, every query goes
    through the LazySearch rounds (tail kernel off), so the round path is what
    the parity cases exercise; the tail kernel has tests of its own."""
    opts.setdefault("tail_queries", 0)
    tree = bkd.bkd_build(P, h, **opts)
    try:
        idx, dist = bkd.bkd_query(tree, Q, k)
        stats = {s: bkd.bkd_get_stat(tree, s) for s in bkd.STATS}
    finally:
        bkd.bkd_free(tree)
    return idx, dist, stats


def test_hand_cases_exact():
    data = json.load(open(GOLDEN))
    for case in data["cases"]:
        P = np.array(case["P"], np.float32)
        for qc in case["queries"]:
            Q = np.array([qc["q"]], np.float32)
            for h in range(0, int(math.log2(P.shape[0])) + 1):
                idx, dist, _ = run(P, Q, qc["k"], h)
                assert idx[0].tolist() == qc["idx"], (case["name"], qc, h)
                assert dist[0].tolist() == [float(x) for x in qc["dist"]]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 10, 11, 16, 20, 27, 32])
def test_every_dimension(d):
    rng = np.random.default_rng(d)
    n = 3000 + d
    P = rng.standard_normal((n, d)).astype(np.float32)
    Q = rng.standard_normal((517, d)).astype(np.float32)
    k = 7
    h = 5
    idx, dist, _ = run(P, Q, k, h)
    check(P, Q, k, idx, dist, oracle.brute_knn(P, Q, k))


@pytest.mark.parametrize("k", [1, 2, 3, 4, 7, 8, 11, 15, 16, 31, 32, 50, 63])
def test_every_list_capacity(k):
    P = workloads.uniform(5000, 6, 7)
    Q = workloads.uniform(700, 6, 8)
    idx, dist, _ = run(P, Q, k, 6)
    check(P, Q, k, idx, dist, oracle.brute_knn(P, Q, k))


@pytest.mark.parametrize("n,h", [(1, 0), (2, 1), (5, 0), (17, 2), (31, 4),
                                 (1000, 9), (4097, 3), (10007, 10)])
def test_ragged_sizes_and_heights(n, h):
    rng = np.random.default_rng(n)
    P = rng.random((n, 3), dtype=np.float32)
    Q = rng.random((300, 3), dtype=np.float32)
    k = min(n, 5)
    idx, dist, _ = run(P, Q, k, h)
    check(P, Q, k, idx, dist, oracle.brute_knn(P, Q, k))


def test_k_equals_n():
    P = workloads.uniform(29, 4, 3)
    Q = workloads.uniform(50, 4, 4)
    idx, dist, _ = run(P, Q, 29 if 29 <= bkd.BKD_MAX_K else 31, 2)
    check(P, Q, 29, idx, dist, oracle.brute_knn(P, Q, 29))


@pytest.mark.parametrize("k", [9, 50])
def test_all_points_identical(k):
    P = np.full((600, 5), 0.25, np.float32)
    Q = np.concatenate([np.full((3, 5), 0.25, np.float32),
                        workloads.uniform(40, 5, 1)])
    idx, dist, stats = run(P, Q, k, 4)
    ref = oracle.brute_knn(P, Q, k)
    check(P, Q, k, idx, dist, ref)
    assert (idx == np.arange(k)).all()   # all tie: smallest indices win
    assert stats["fallback"] == Q.shape[0]


def test_integer_grid_ties():
    rng = np.random.default_rng(12)
    P = rng.integers(0, 5, (4000, 3)).astype(np.float32)
    Q = (rng.integers(-2, 12, (1000, 3)) * 0.5).astype(np.float32)
    for k in (1, 6, 20):
        idx, dist, stats = run(P, Q, k, 6)
        check(P, Q, k, idx, dist, oracle.brute_knn(P, Q, k))


def test_duplicates_and_queries_on_points():
    P = workloads.with_duplicates(workloads.uniform(8000, 10, 5), 0.05, 2)
    Q = np.concatenate([P[::97], workloads.uniform(500, 10, 6)])
    idx, dist, _ = run(P, Q, 10, 7)
    check(P, Q, 10, idx, dist, oracle.brute_knn(P, Q, 10))


def test_far_queries_and_tiny_scales():
    rng = np.random.default_rng(21)
    P = (rng.standard_normal((3000, 4)) * 1e-6).astype(np.float32)
    Q = np.concatenate([
        (rng.standard_normal((100, 4)) * 1e-6).astype(np.float32),
        (rng.standard_normal((100, 4)) * 1e3).astype(np.float32)])
    idx, dist, _ = run(P, Q, 5, 5)
    check(P, Q, 5, idx, dist, oracle.brute_knn(P, Q, 5))


def test_uniform_65536_full_queryset():
    """n=65,536, m=16,384, d=10, uniform [0,1)^10 (seeds 0 / 1), k=10,
    height 8 (256 leaves of 256 points): every query against brute force."""
    w = workloads.UNIFORM_64K
    P, Q = w.points(), w.queries()
    idx, dist, stats = run(P, Q, w.k, w.height, tail_queries=-1)
    info = check(P, Q, w.k, idx, dist, oracle.brute_knn(P, Q, w.k))
    assert stats["rounds"] >= 2 and stats["pairs"] > 0
    print("uniform 64K:", info, stats)


def test_mixture_scaled():
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 20, 1 << 15, 10)
    P, Q = w.points(), w.queries()
    idx, dist, stats = run(P, Q, w.k, w.height, tail_queries=-1)
    rows = np.arange(0, Q.shape[0], 4)
    ref = oracle.brute_knn(P, Q[rows], w.k)
    print("mixture 2^20:", check(P, Q, w.k, idx, dist, ref, rows), stats)


def test_tree_matches_oracle_tree():
    """The library's median-split tree equals the oracle's (same rule,
    independent code): split values, leaf bounds and leaf membership."""
    P = workloads.mixture(20000, workloads.mixture_params(7, 8, .05, .2, 0), 3)
    for h in (0, 3, 8):
        tree = bkd.bkd_build(P, h)
        split, leaf_lo, perm = bkd.bkd_export_tree(tree)
        bkd.bkd_free(tree)
        ot = oracle.build_tree(P, h)
        assert np.array_equal(leaf_lo, ot.leaf_lo)
        assert np.array_equal(split, ot.split[:len(split)])
        sizes = np.diff(leaf_lo)
        mine = np.empty(P.shape[0], np.int64)
        mine[perm] = np.repeat(np.arange(1 << h), sizes)
        assert np.array_equal(mine, ot.leaf_of_point())


@pytest.mark.parametrize("chunks", [1, 2, 3, 10])
def test_chunked_mode_is_bit_identical(chunks):
    """Streaming the leaf structure in N leaf chunks (Sec. 3.2) changes only
    the schedule: results equal the resident run bit for bit."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 17, 1 << 13, 9)
    P, Q = w.points(), w.queries()
    idx0, dist0, _ = run(P, Q, w.k, w.height)
    idx1, dist1, st = run(P, Q, w.k, w.height, chunks=chunks)
    assert np.array_equal(idx0, idx1) and np.array_equal(dist0, dist1)
    if chunks > 2:
        assert st["chunk_bytes"] > 0
    check(P, Q, w.k, idx1, dist1, oracle.brute_knn(P, Q[:512], w.k),
          rows=np.arange(512))


@pytest.mark.parametrize("chunks", [1, 2, 3, 10])
def test_bf16_screen_in_chunked_mode_is_bit_identical(chunks):
    """The warp screen on a chunked tree: each chunk's screen operands are
    copied with its points and the screen runs on the chunk buffers; the
    result equals the resident float32 path, and the copies include the
    screen operands."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 17, 8000, 9)
    P, Q = w.points(), w.queries()
    tree = bkd.bkd_build(P, w.height)
    i0, d0 = bkd.bkd_query(tree, Q, w.k)
    bkd.bkd_free(tree)
    tree = bkd.bkd_build(P, w.height, precision=1, chunks=chunks,
                         tail_queries=0)
    try:
        # float32 first: the chunks it leaves resident carry no screen
        # operands yet, the screened call must bring them in
        bkd.bkd_set_option(tree, "precision", 0)
        i2, d2 = bkd.bkd_query(tree, Q, w.k)
        st0 = {s: bkd.bkd_get_stat(tree, s) for s in bkd.STATS}
        bkd.bkd_set_option(tree, "precision", 1)
        i1, d1 = bkd.bkd_query(tree, Q, w.k)
        st = {s: bkd.bkd_get_stat(tree, s) for s in bkd.STATS}
    finally:
        bkd.bkd_free(tree)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    assert np.array_equal(i0, i2) and np.array_equal(d0, d2)
    assert st["screen_pairs"] > 0 and st0["screen_pairs"] == 0
    assert st["screen_kept"] < 0.5 * st["screen_pairs"]
    # the screen operands (32 B per point and k-half) travel with the points
    # (N = 1: the single chunk stays resident, only its operands are copied)
    assert st["chunk_bytes"] > 0
    check(P, Q, w.k, i1, d1, oracle.brute_knn(P, Q[:500], w.k),
          rows=np.arange(500))


@pytest.mark.parametrize("chunks", [2, 3, 7])
def test_point_split_chunks_are_bit_identical(chunks):
    """The paper's point chunks (Sec. 3.2: positions ceil(j n / N) .. of the
    leaf structure, so leaves straddle chunks and their queries are scanned
    piecewise in consecutive chunks) give the same results as the resident
    tree; n is not a multiple of the chunk count or of 4."""
    w = workloads.scaled(workloads.MIXTURE_64M, (1 << 17) + 1237, 1 << 13, 9)
    P, Q = w.points(), w.queries()
    idx0, dist0, _ = run(P, Q, w.k, w.height)
    idx1, dist1, st = run(P, Q, w.k, w.height, chunks=chunks, point_chunks=1)
    assert np.array_equal(idx0, idx1) and np.array_equal(dist0, dist1)
    assert st["chunk_bytes"] > 0
    check(P, Q, w.k, idx1, dist1, oracle.brute_knn(P, Q[:512], w.k),
          rows=np.arange(512))


def test_chunk_schedule_streams_less_than_every_chunk_every_round():
    """Leaf-aligned chunks keep the resident chunks running while they hold
    buffered queries: far fewer bytes are copied than one pass over the
    leaf structure per round, and the results stay those of the resident
    tree."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 18, 1 << 14, 10)
    P, Q = w.points(), w.queries()
    idx0, dist0, _ = run(P, Q, w.k, w.height)
    tree = bkd.bkd_build(P, w.height, chunks=8, tail_queries=0)
    try:
        idx1, dist1 = bkd.bkd_query(tree, Q, w.k)
        rounds = bkd.bkd_get_stat(tree, "rounds")
        copied = bkd.bkd_get_stat(tree, "chunk_bytes")
    finally:
        bkd.bkd_free(tree)
    assert np.array_equal(idx0, idx1) and np.array_equal(dist0, dist1)
    structure = (1 << 18) * 10 * 4  # the leaf structure's float32 points
    assert copied < 0.5 * rounds * structure, (copied, rounds)


def test_chunked_by_memory_cap():
    P = workloads.uniform(50000, 10, 1)
    Q = workloads.uniform(3000, 10, 2)
    tree = bkd.bkd_build(P, 7, device_mem_cap=400_000)
    shape = bkd.bkd_tree_shape(tree)
    idx, dist = bkd.bkd_query(tree, Q, 10)
    bkd.bkd_free(tree)
    assert shape["chunked"] and shape["chunks"] >= 2
    check(P, Q, 10, idx, dist, oracle.brute_knn(P, Q, 10))


def test_query_slicing_is_bit_identical():
    P = workloads.uniform(30000, 8, 3)
    Q = workloads.uniform(5000, 8, 4)
    idx0, dist0, _ = run(P, Q, 10, 7)
    idx1, dist1, _ = run(P, Q, 10, 7, max_active=777)
    assert np.array_equal(idx0, idx1) and np.array_equal(dist0, dist1)


def test_device_pointers_and_streams():
    torch = pytest.importorskip("torch")
    P = workloads.uniform(20000, 10, 1)
    Q = workloads.uniform(3000, 10, 2)
    Pd = torch.from_numpy(P).cuda()
    Qd = torch.from_numpy(Q).cuda()
    tree = bkd.bkd_build(Pd, 6)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        idx, dist = bkd.bkd_query(tree, Qd, 10)
    s.synchronize()
    assert idx.is_cuda and dist.is_cuda
    idx_h, dist_h = bkd.bkd_query(tree, Q, 10)
    bkd.bkd_free(tree)
    assert np.array_equal(idx.cpu().numpy(), idx_h)
    check(P, Q, 10, idx_h, dist_h, oracle.brute_knn(P, Q, 10))


def test_rejects_non_finite_queries_and_stays_usable():
    P = workloads.uniform(2000, 3, 1)
    tree = bkd.bkd_build(P, 3)
    Q = workloads.uniform(10, 3, 2)
    Q[4, 1] = np.nan
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_query(tree, Q, 3)
    assert e.value.code == bkd.BKD_EINVAL
    Q[4, 1] = 0.5
    idx, dist = bkd.bkd_query(tree, Q, 3)
    bkd.bkd_free(tree)
    check(P, Q, 3, idx, dist, oracle.brute_knn(P, Q, 3))


def test_empty_query_set_and_bad_k():
    P = workloads.uniform(100, 2, 1)
    tree = bkd.bkd_build(P, 2)
    idx, dist = bkd.bkd_query(tree, np.zeros((0, 2), np.float32), 4)
    assert idx.shape == (0, 4)
    with pytest.raises(bkd.BkdError):
        bkd.bkd_query(tree, np.zeros((3, 2), np.float32), 101)
    bkd.bkd_free(tree)


@pytest.mark.parametrize("kind", ["uniform", "mixture"])
def test_tail_kernel_is_bit_identical(kind):
    """Finishing the last queries in one launch (one warp per query) instead
    of one LazySearch round per leaf changes only the schedule."""
    if kind == "uniform":
        P, Q = workloads.uniform(60000, 10, 1), workloads.uniform(6000, 10, 2)
    else:
        w = workloads.scaled(workloads.MIXTURE_64M, 1 << 17, 6000, 7)
        P, Q = w.points(), w.queries()
    res = {}
    for tail in (0, 500, -1, 10 ** 6):
        idx, dist, st = run(P, Q, 10, 7, tail_queries=tail)
        res[tail] = (idx, dist, st)
    base_i, base_d, base_st = res[0]
    assert base_st["tail_queries"] == 0
    assert res[10 ** 6][2]["tail_queries"] == Q.shape[0]
    assert res[10 ** 6][2]["rounds"] == 0
    for tail, (i, dd, st) in res.items():
        assert np.array_equal(i, base_i) and np.array_equal(dd, base_d), tail
    check(P, Q, 10, base_i, base_d, oracle.brute_knn(P, Q[:1000], 10),
          rows=np.arange(1000))


@pytest.mark.parametrize("k", [31, 32, 40, 63])
def test_tail_kernel_long_lists(k):
    """Lists of 33..64 entries take two entries per lane in the tail kernel;
    the result equals the round-by-round path bit for bit."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 16, 3000, 7)
    P, Q = w.points(), w.queries()
    i0, d0, _ = run(P, Q, k, 7, tail_queries=0)
    i1, d1, st = run(P, Q, k, 7, tail_queries=10 ** 6)
    assert st["tail_queries"] == Q.shape[0]
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    check(P, Q, k, i1, d1, oracle.brute_knn(P, Q[:300], k),
          rows=np.arange(300))


@pytest.mark.parametrize("chunks", [1, 2, 3, 10])
def test_tail_kernel_in_chunked_mode(chunks):
    """The tail kernel on a chunked tree reads the leaves of the two
    resident chunk buffers there and the others from the mapped host copy
    (N <= 2: nothing mapped)."""
    w = workloads.scaled(workloads.MIXTURE_64M, 1 << 16, 3000, 8)
    P, Q = w.points(), w.queries()
    i0, d0, _ = run(P, Q, 10, 8, tail_queries=0)
    i1, d1, st = run(P, Q, 10, 8, chunks=chunks, tail_queries=1500)
    assert st["tail_queries"] > 0
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    if chunks <= 2:
        # only the re-check's few binary64 rows (and the fallback) read
        # mapped memory
        assert st["mapped_bytes"] < 0.01 * st["tail_pairs"] * 4 * 10


def run_both_precisions(P, Q, k, h, **opts):
    """One tree with the screen data of both BF16 screen kernels; the same
    queries scored with the float32 kernel only, with the warp screen
    kernel and with the tcgen05 screen kernel.  The two screens must agree
    with each other bit for bit; returns the float32 result, the warp
    screen's result and the stats of both screens."""
    opts.setdefault("tail_queries", 0)
    tree = bkd.bkd_build(P, h, precision=1, screen_kernel=2, **opts)
    try:
        bkd.bkd_set_option(tree, "precision", 0)
        i0, d0 = bkd.bkd_query(tree, Q, k)
        bkd.bkd_set_option(tree, "precision", 1)
        out = []
        for kernel in (0, 1):
            bkd.bkd_set_option(tree, "screen_kernel", kernel)
            i1, d1 = bkd.bkd_query(tree, Q, k)
            out.append((i1, d1,
                        {s: bkd.bkd_get_stat(tree, s) for s in bkd.STATS}))
    finally:
        bkd.bkd_free(tree)
    (i1, d1, st), (i2, d2, st2) = out
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2), \
        "the warp and tcgen05 screen kernels disagree"
    return i0, d0, i1, d1, (st, st2)


@pytest.mark.parametrize("d,k", [(2, 4), (3, 10), (10, 10), (10, 1), (10, 31),
                                 (16, 10), (17, 10), (27, 5), (32, 10),
                                 (27, 50), (10, 63)])
def test_bf16_screen_is_bit_identical(d, k):
    """The BF16 tensor-core screen only skips points that provably cannot
    enter a list; survivors are scored in float32, so results equal the
    float32 path bit for bit."""
    params = workloads.mixture_params(d, 16, 0.02, 0.2, 0)
    P = workloads.mixture(60000, params, 1)
    Q = workloads.mixture(4000, params, 2)
    i0, d0, i1, d1, sts = run_both_precisions(P, Q, k, 7)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    for st in sts:
        assert st["screen_pairs"] > 0
        # (the tcgen05 kernel counts a kept (point, 16-query group) as 16)
        assert st["screen_kept"] < 0.5 * st["screen_pairs"]
    check(P, Q, k, i1, d1, oracle.brute_knn(P, Q[:600], k),
          rows=np.arange(600))


def test_bf16_screen_with_ties_and_duplicates():
    rng = np.random.default_rng(4)
    P = rng.integers(0, 6, (20000, 4)).astype(np.float32)
    Q = (rng.integers(-2, 14, (2000, 4)) * 0.5).astype(np.float32)
    i0, d0, i1, d1, _ = run_both_precisions(P, Q, 10, 6)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    Pd = workloads.with_duplicates(workloads.uniform(30000, 10, 5), 0.05, 2)
    Qd = np.concatenate([Pd[::50], workloads.uniform(1000, 10, 6)])
    i0, d0, i1, d1, _ = run_both_precisions(Pd, Qd, 10, 7)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    check(Pd, Qd, 10, i1, d1, oracle.brute_knn(Pd, Qd, 10))


def test_bf16_screen_uniform_65536():
    w = workloads.UNIFORM_64K
    P, Q = w.points(), w.queries()
    i0, d0, i1, d1, sts = run_both_precisions(P, Q, w.k, w.height,
                                              tail_queries=-1)
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    check(P, Q, w.k, i1, d1, oracle.brute_knn(P, Q, w.k))
    for st in sts:
        print("screen kept fraction", st["screen_kept"] / st["screen_pairs"])


def test_bf16_screen_option_errors():
    P = workloads.uniform(5000, 4, 1)
    tree = bkd.bkd_build(P, 4)
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_set_option(tree, "precision", 1)
    assert e.value.code == bkd.BKD_EINVAL
    bkd.bkd_free(tree)
    # a screen kernel whose layout the tree does not hold, and item sizes
    # outside the selected kernel's range
    for built, other in ((0, 1), (1, 0)):
        tree = bkd.bkd_build(P, 4, precision=1, screen_kernel=built)
        try:
            with pytest.raises(bkd.BkdError) as e:
                bkd.bkd_set_option(tree, "screen_kernel", other)
            assert e.value.code == bkd.BKD_EINVAL
            bad = 64 if built == 0 else 8
            with pytest.raises(bkd.BkdError) as e:
                bkd.bkd_set_option(tree, "screen_tile", bad)
            assert e.value.code == bkd.BKD_EINVAL
        finally:
            bkd.bkd_free(tree)
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_build(P, 4, precision=1, screen_kernel=3)
    assert e.value.code == bkd.BKD_EINVAL
    # chunked trees: the screen needs leaf chunks and the warp kernel
    for opts in ({"point_chunks": 1}, {"screen_kernel": 1}):
        with pytest.raises(bkd.BkdError) as e:
            bkd.bkd_build(P, 4, precision=1, chunks=2, **opts)
        assert e.value.code == bkd.BKD_EUNSUPPORTED


def test_d27_k50_duplicates_workload():
    """The d = 27, k = 50 workload (64-component mixture, 1% of the rows
    exact copies of others) at a size the oracle finishes: default options
    (tail kernel automatic, its lists of k + 1 = 51 entries two per lane)
    and the BF16 screen, both against the oracle."""
    w = workloads.scaled(workloads.MIXTURE_D27, 1 << 16, 2000, 8)
    P, Q = w.points(), w.queries()
    ref = oracle.brute_knn(P, Q, 50)
    tree = bkd.bkd_build(P, w.height, precision=1, screen_kernel=2)
    try:
        for prec, kernel in ((0, 0), (1, 0), (1, 1)):
            bkd.bkd_set_option(tree, "precision", prec)
            bkd.bkd_set_option(tree, "screen_kernel", kernel)
            idx, dist = bkd.bkd_query(tree, Q, 50)
            check(P, Q, 50, idx, dist, ref)
            assert bkd.bkd_get_stat(tree, "tail_queries") > 0
    finally:
        bkd.bkd_free(tree)
