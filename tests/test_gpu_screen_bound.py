"""The BF16 screen's safety bound, attacked where it is thinnest (needs a GPU).

The screen (ProcessAllBuffers with bf16 tensor cores, float32 rescoring) may
only skip points that provably cannot enter a candidate list, so its results
must equal the float32 path bit for bit and the binary64 oracle.  The bound
has three ingredients, each attacked here:

  * bf16 rounding of the centred coordinates (8 significant bits: relative
    error up to 2^-8): a hand-built case whose query and point offsets sit
    just beyond / just short of a bf16 rounding tie, so that rounding moves
    them apart by almost the full 2^-8 of each, and whose (k+1)-th bound is
    just above the point's distance.  A bound that assumed 2^-9 rejects the
    point (worked through in the test's docstring);
  * the tensor core's fp32 accumulation: the probe entry points run the
    warp kernel's mma.sync m16n8k16 and the tcgen05 kernel's path (its
    operand layout, descriptors and chained MMAs) on adversarial operands
    and every result is compared with the exact sum against the
    accumulation model the bound uses (error <= 2^-18 of the sum of
    absolute terms per MMA k-step);
  * wide data: a large common offset, queries far outside the tree's box,
    leaves of tiny spread, and d = 17 / 32 (two and three k-halves).
"""
import math

import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads
from parity import check

pytestmark = pytest.mark.gpu

MODEL = 2.0 ** -18   # per-instruction accumulation error the bound assumes


def run_both(P, Q, k, h):
    """float32 path and both BF16 screen kernels on one tree, every query
    through the LazySearch rounds (tail kernel off); the two screens must
    agree bit for bit.  Returns the float32 and warp-screen results and the
    stats of the tcgen05 screen's call (screen_pairs of both are equal)."""
    tree = bkd.bkd_build(P, h, precision=1, screen_kernel=2, tail_queries=0)
    try:
        bkd.bkd_set_option(tree, "precision", 0)
        i0, d0 = bkd.bkd_query(tree, Q, k)
        bkd.bkd_set_option(tree, "precision", 1)
        i1, d1 = bkd.bkd_query(tree, Q, k)
        bkd.bkd_set_option(tree, "screen_kernel", 1)
        i2, d2 = bkd.bkd_query(tree, Q, k)
        st = {s: bkd.bkd_get_stat(tree, s) for s in bkd.STATS}
    finally:
        bkd.bkd_free(tree)
    assert np.array_equal(i1, i2) and np.array_equal(d1, d2), \
        "the warp and tcgen05 screen kernels disagree"
    return i0, d0, i1, d1, st


# ------------------------------------------------------------ rounding case
def rounding_case(scale: float, d: int, mirror: bool):
    """Two leaves split on x0 at 0.  Leaf A (x0 < 0) has the bounding box
    [-2, -1e-3] x [-9.0312, 9.0312], centre (-1.0005, 0); leaf B holds the
    query's two nearest rivals at distances 1.0002 and 1.0003.  The query
    q = (0, 10.0313) lies in B, so the first (float32) round fills its k+1 =
    2 list from B (bound 1.0003^2) and the second round screens A.  A's point
    x = (-1e-3, 9.0312) is at distance 1.0001 < 1.0003, so it must enter.
    Centred: v = (1.0005, 10.0313) -> bf16 (1, 10.0625) (10.0313 is past the
    tie 10.03125), w = (0.9995, 9.0312) -> bf16 (1, 9) (9.0312 is short of
    the tie 9.03125): |v^ - w^| = 1.0625, although |q - x| = 1.0001.  With
    rho = 2^-8 the screen's threshold radius is ~1.0807 and keeps x; with
    2^-9 it is ~1.0432 and x would be lost (query answered with B's point).
    Scaling by a power of two keeps every rounding; extra dimensions are
    zero (d = 17 / 32 use two / three k-halves)."""
    base = np.array([
        [-2.0, -9.0312], [-2.0, 9.0312], [-1e-3, 9.0312], [-1.5, 0.0],
        [0.0, 11.0315], [0.0, 11.0316], [2.0, 30.0], [1.0, -30.0]],
        np.float32)
    q = np.array([[0.0, 10.0313]], np.float32)
    if mirror:
        base[:, 1] *= -1
        q[:, 1] *= -1
    P = np.zeros((8, d), np.float32)
    Q = np.zeros((1, d), np.float32)
    P[:, :2] = base * np.float32(scale)
    Q[:, :2] = q * np.float32(scale)
    return P, Q


@pytest.mark.parametrize("d", [2, 17, 32])
@pytest.mark.parametrize("scale", [2.0 ** -8, 1.0, 2.0 ** 6])
@pytest.mark.parametrize("mirror", [False, True])
def test_screen_keeps_point_moved_apart_by_bf16_rounding(d, scale, mirror):
    P, Q = rounding_case(scale, d, mirror)
    ref = oracle.brute_knn(P, Q, 1)
    assert ref.idx[0, 0] == 2          # the point of leaf A is the answer
    i0, d0, i1, d1, st = run_both(P, Q, 1, 1)
    assert st["screen_pairs"] > 0      # leaf A went through the screen
    assert i0[0, 0] == 2 and i1[0, 0] == 2, (i0, i1)
    assert np.array_equal(d0, d1)
    check(P, Q, 1, i1, d1, ref)


# -------------------------------------------------------- accumulation model
def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even bf16 bit patterns of float32 values."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_value(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b).astype(np.uint32) << 16).view(np.float32) \
        .astype(np.float64)


def exact_dots(A, Bt):
    """Exact A Bt^T per instance with math.fsum (bf16 products are exact in
    binary64; fsum rounds the exact sum once) and the sums of the absolute
    products."""
    a, b = bf16_value(A), bf16_value(Bt)
    cnt, rows, _ = a.shape
    n = b.shape[1]
    out = np.empty((cnt, rows, n))
    mag = np.einsum("irk,ick->irc", np.abs(a), np.abs(b))
    for i in range(cnt):
        prod = a[i][:, None, :] * b[i][None, :, :]
        for r in range(rows):
            for c in range(n):
                out[i, r, c] = math.fsum(prod[r, c])
    return out, mag


def adversarial_operands(rng, cnt, n, kh):
    """Instances of four kinds: (0) one large product with small same-sign
    ones just under its last bits, so that truncating alignment would lose
    them all in the same direction; (1) heavy cancellation: pairs of equal
    and opposite large products plus small terms; (2) exponents mixed over
    2^-15..2^15 inside each k-half; (3) the screen's own rows and columns:
    centred offsets, the norm split against -1/2 and a threshold split into
    three bf16 parts."""
    K = 16 * kh
    A = np.zeros((cnt, 128, K), np.float32)
    B = np.zeros((cnt, n, K), np.float32)
    for i in range(cnt):
        kind = i % 4
        if kind == 0:
            A[i] = rng.uniform(1.0, 2.0, (128, K))
            B[i] = rng.uniform(1.0, 2.0, (n, K))
            big = 2.0 ** rng.integers(8, 12)
            A[i][:, 0] *= big
            B[i][:, 0] *= big
            A[i][:, 1:] *= 2.0 ** -rng.integers(6, 10, (128, K - 1))
        elif kind == 1:
            half = K // 2
            x = rng.uniform(1.0, 2.0, (128, half)) * 2.0 ** rng.integers(4, 10)
            A[i][:, :half] = x
            A[i][:, half:] = -x
            B[i][:] = 1.0
            A[i][:, K - 1] = rng.uniform(-1e-3, 1e-3, 128)
            B[i][:, half - 1] = rng.uniform(1.0, 1.1, n)
        elif kind == 2:
            A[i] = (rng.choice([-1, 1], (128, K)) * rng.uniform(1, 2, (128, K))
                    * 2.0 ** rng.integers(-15, 15, (128, K)))
            B[i] = (rng.choice([-1, 1], (n, K)) * rng.uniform(1, 2, (n, K))
                    * 2.0 ** rng.integers(-15, 15, (n, K)))
        else:
            d = K - 5
            sc = 2.0 ** rng.integers(-4, 4)
            w = bf16_value(bf16_bits((rng.standard_normal((128, d)) * sc)
                                     .astype(np.float32)))
            pn = (w ** 2).sum(1).astype(np.float32)
            hi = bf16_value(bf16_bits(pn))
            lo = bf16_value(bf16_bits((pn - hi).astype(np.float32)))
            A[i][:, :d] = w
            A[i][:, d] = hi
            A[i][:, d + 1] = lo
            A[i][:, d + 2:d + 5] = 1.0
            v = rng.standard_normal((n, d)) * sc
            t = (rng.uniform(0.5, 2.0, n) * (v ** 2).sum(1)).astype(np.float32)
            th = bf16_value(bf16_bits(t))
            tm = bf16_value(bf16_bits((t - th).astype(np.float32)))
            tl = bf16_value(bf16_bits((t - th - tm).astype(np.float32)))
            B[i][:, :d] = v
            B[i][:, d] = -0.5
            B[i][:, d + 1] = -0.5
            B[i][:, d + 2], B[i][:, d + 3], B[i][:, d + 4] = th, tm, tl
    return bf16_bits(A), bf16_bits(B)


@pytest.mark.parametrize("n,kh", [(16, 1), (48, 1), (128, 1), (32, 2),
                                  (128, 3)])
def test_tensor_core_accumulation_within_the_screen_model(n, kh):
    """Every result of the screen's tcgen05 path is within kh 2^-18 of the
    sum of its absolute products from the exact sum (the model of the
    bound); also checks the operand layout and descriptors (a wrong layout
    gives wrong sums, far outside the model)."""
    rng = np.random.default_rng(2024 + n + kh)
    A, Bt = adversarial_operands(rng, 8, n, kh)
    D = bkd.bkd_probe_umma(A, Bt)
    exact, mag = exact_dots(A, Bt)
    err = np.abs(D.astype(np.float64) - exact)
    ratio = err / np.maximum(mag, 1e-300)
    worst = float(ratio.max())
    print(f"n={n} kh={kh}: accumulation error / sum |a b|: max {worst:.3e}"
          f" = 2^{math.log2(worst) if worst > 0 else -math.inf:.2f}; "
          f"model {kh} x 2^-18")
    assert np.isfinite(D).all()
    assert worst <= kh * MODEL, f"accumulation error {worst:.3e}"


def test_tensor_core_padding_rows_and_columns():
    """A padding point (pn_hi = +inf against the query's -1/2) gives -inf,
    never NaN, also against a column whose threshold is +2^126 (list not
    full); a padding column (threshold -2^126) gives a large negative value
    against every real point."""
    rng = np.random.default_rng(3)
    d = 10
    A = np.zeros((1, 128, 16), np.float32)
    B = np.zeros((1, 16, 16), np.float32)
    A[0, :, :d] = rng.standard_normal((128, d))
    A[0, :, d] = 1.0
    A[0, :, d + 2:d + 5] = 1.0
    A[0, 100:, :] = 0.0
    A[0, 100:, d] = np.inf
    B[0, :, :d] = rng.standard_normal((16, d))
    B[0, :, d:d + 2] = -0.5
    B[0, :8, d + 2] = 2.0 ** 126
    B[0, 8:12, d + 2] = -(2.0 ** 126)
    D = bkd.bkd_probe_umma(bf16_bits(A), bf16_bits(B))[0]
    assert (D[100:] == -np.inf).all()
    assert (D[:100, :8] > 2.0 ** 125).all()
    assert (D[:100, 8:12] < -(2.0 ** 125)).all()
    assert np.isfinite(D[:100]).all()


# ----------------------------- accumulation model, warp kernel (mma.sync)
def mma_exact_dots(A, Bt, C):
    """Exact C + A Bt^T per instance with math.fsum (bf16 products are exact
    in binary64; fsum rounds the exact sum once), and the sum of absolute
    terms."""
    a, b = bf16_value(A), bf16_value(Bt)
    cnt = A.shape[0]
    out = np.empty((cnt, 16, 8))
    mag = np.empty((cnt, 16, 8))
    for i in range(cnt):
        prod = a[i][:, None, :] * b[i][None, :, :]      # 16 x 8 x 16
        for r in range(16):
            for c in range(8):
                terms = list(prod[r, c]) + [float(C[i, r, c])]
                out[i, r, c] = math.fsum(terms)
                mag[i, r, c] = math.fsum(abs(t) for t in terms)
    return out, mag


def mma_adversarial_operands(rng, cnt):
    """Instances of several kinds (a quarter each): one large product with
    fifteen small same-sign ones just under the large one's last bits;
    heavy cancellation (pairs of equal and opposite large products) with
    small terms; exponents mixed over 2^-30..2^30 inside one k-half; the
    screen's own shape (offsets, the norm split pn_hi / pn_lo against -1/2,
    a large accumulator input)."""
    A = np.zeros((cnt, 16, 16), np.float32)
    B = np.zeros((cnt, 8, 16), np.float32)
    C = np.zeros((cnt, 16, 8), np.float32)
    for i in range(cnt):
        kind = i % 4
        if kind == 0:
            A[i] = rng.uniform(1.0, 2.0, (16, 16))
            B[i] = rng.uniform(1.0, 2.0, (8, 16))
            big = 2.0 ** rng.integers(8, 12)
            A[i][:, 0] *= big
            B[i][:, 0] *= big
            small = 2.0 ** -rng.integers(6, 10, (16, 15))
            A[i][:, 1:] *= small
        elif kind == 1:
            x = rng.uniform(1.0, 2.0, (16, 8)) * 2.0 ** rng.integers(4, 10)
            A[i][:, 0:8] = x
            A[i][:, 8:16] = -x
            B[i][:] = 1.0
            A[i][:, 15] = rng.uniform(-1e-3, 1e-3, 16)
            B[i][:, 7] = rng.uniform(1.0, 1.1, 8)
        elif kind == 2:
            A[i] = (rng.choice([-1, 1], (16, 16)) * rng.uniform(1, 2, (16, 16))
                    * 2.0 ** rng.integers(-15, 15, (16, 16)))
            B[i] = (rng.choice([-1, 1], (8, 16)) * rng.uniform(1, 2, (8, 16))
                    * 2.0 ** rng.integers(-15, 15, (8, 16)))
            C[i] = rng.standard_normal((16, 8)) * 2.0 ** rng.integers(-10, 10)
        else:
            d = 10
            w = rng.standard_normal((16, d)) * 2.0 ** rng.integers(-4, 4)
            wb = bf16_value(bf16_bits(w.astype(np.float32)))
            pn = np.float32((wb ** 2).sum(1))
            hi = bf16_value(bf16_bits(pn))
            lo = bf16_value(bf16_bits((pn - hi).astype(np.float32)))
            A[i][:, :d] = w
            A[i][:, d] = hi
            A[i][:, d + 1] = lo
            v = rng.standard_normal((8, d)) * 2.0 ** rng.integers(-4, 4)
            B[i][:, :d] = v
            B[i][:, d] = -0.5
            B[i][:, d + 1] = -0.5
            C[i] = rng.standard_normal((16, 8)) * 4.0
    return bf16_bits(A), bf16_bits(B), C


def test_mma_sync_accumulation_within_the_screen_model():
    """The warp screen kernel's mma.sync m16n8k16 on adversarial operands:
    every result within 2^-18 of |c| + sum |a b| from the exact sum."""
    rng = np.random.default_rng(2024)
    A, Bt, C = mma_adversarial_operands(rng, 512)
    D = bkd.bkd_probe_mma(A, Bt, C)
    exact, mag = mma_exact_dots(A, Bt, C)
    err = np.abs(D.astype(np.float64) - exact)
    ratio = err / np.maximum(mag, 1e-300)
    worst = float(ratio.max())
    print(f"accumulation error / (|c| + sum |a b|): max {worst:.3e} "
          f"= 2^{math.log2(worst) if worst > 0 else -math.inf:.2f}; "
          f"model 2^-18")
    assert np.isfinite(D).all()
    assert worst <= MODEL, f"accumulation error {worst:.3e} exceeds 2^-18"


def test_mma_sync_infinite_norm_slot_gives_minus_infinity():
    """A padding point carries pn_hi = +inf against the query's -1/2: its
    product must be -inf, never NaN, whatever the other slots hold."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((1, 16, 16)).astype(np.float32)
    B = rng.standard_normal((1, 8, 16)).astype(np.float32)
    A[0, :, 12] = np.inf
    B[0, :, 12] = -0.5
    C = rng.standard_normal((1, 16, 8)).astype(np.float32)
    D = bkd.bkd_probe_mma(bf16_bits(A), bf16_bits(B), C)
    assert (D == -np.inf).all()


# ------------------------------------------------------------- wide data
def _screen_vs_oracle(P, Q, k, h, rows=600):
    i0, d0, i1, d1, st = run_both(P, Q, k, h)
    assert st["screen_pairs"] > 0
    assert np.array_equal(i0, i1) and np.array_equal(d0, d1)
    sel = np.arange(min(rows, Q.shape[0]))
    check(P, Q, k, i1, d1, oracle.brute_knn(P, Q[sel], k), rows=sel)
    return st


@pytest.mark.parametrize("d", [10, 17, 32])
def test_screen_large_common_offset(d):
    """Every coordinate offset by 1e3: centring removes the offset, but the
    points carry float32 quantisation of ~6e-5 at that magnitude."""
    params = workloads.mixture_params(d, 16, 0.02, 0.2, 0)
    P = workloads.mixture(50000, params, 1) + np.float32(1000.0)
    Q = workloads.mixture(3000, params, 2) + np.float32(1000.0)
    _screen_vs_oracle(P, Q, 10, 7)


@pytest.mark.parametrize("d", [10, 17, 32])
def test_screen_far_queries(d):
    """Queries far outside the tree's bounding box (shifted by 3 and by up
    to 1e3 in some coordinates): |v^| is large against the leaf, where the
    accumulation term E is largest relative to the threshold."""
    rng = np.random.default_rng(d)
    params = workloads.mixture_params(d, 16, 0.02, 0.2, 0)
    P = workloads.mixture(50000, params, 1)
    Q = workloads.mixture(3000, params, 2)
    Q[:1000] += np.float32(3.0)
    far = rng.choice(d, (1000, 2))
    Q[np.arange(1000, 2000)[:, None], far] += rng.choice(
        [-1e3, 1e3], (1000, 2)).astype(np.float32)
    _screen_vs_oracle(P, Q, 10, 7, rows=Q.shape[0])


@pytest.mark.parametrize("d", [4, 17, 32])
def test_screen_tiny_spread_leaves(d):
    """64 clusters of spread 1e-4: leaves whose points differ in the last
    bits of their float32 coordinates."""
    params = workloads.mixture_params(d, 64, 1e-4, 1e-4, 3)
    P = workloads.mixture(40000, params, 1)
    Q = workloads.mixture(3000, params, 2)
    _screen_vs_oracle(P, Q, 8, 8)
