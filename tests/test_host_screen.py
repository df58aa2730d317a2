"""The host half of bkd_build, checked without a GPU (bkd_test_host_screen):
the median-split tree against the oracle's (Sec. 2.3), the node bounding
boxes against their definition, and the BF16 screens' operands (the warp
kernel's fragments and the tcgen05 kernel's tiles) and per-leaf bounds
against exact rational arithmetic.

The screen drops a point only if a bound that uses these host values says it
cannot enter the list, so the host half of that bound is pinned here on data
built to stress it: offsets from the leaf centre just below and at bf16
rounding ties, mixed exponents inside one point, a large common offset,
leaves of tiny spread and float32 subnormals.  A bound that took bf16's
rounding error as 2^-9 instead of 2^-8 fails on the tie data (checked).  On
the subnormal data the norm split loses pn entirely (it underflows), which
is why a leaf's pn_max is floored: the screen's error term E then holds an
absolute 2^-100 that covers every underflow error.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import paper_1512_02831_gb300 as bkd
import workloads

TWO = Fraction(2)


def bf16_nearest_even(f32: np.ndarray) -> np.ndarray:
    """bf16 bit patterns of float32 values: the nearer of the two
    neighbouring bf16 values (compared in float64, exact here), the one with
    an even last bit on a tie."""
    b = np.ascontiguousarray(f32, np.float32).view(np.uint32)
    lo = b & np.uint32(0xFFFF0000)            # toward zero
    hi = lo + np.uint32(0x10000)              # away from zero
    x = b.view(np.float32).astype(np.float64)
    dlo = np.abs(x - lo.view(np.float32).astype(np.float64))
    dhi = np.abs(hi.view(np.float32).astype(np.float64) - x)
    odd = ((lo >> np.uint32(16)) & np.uint32(1)) == 1
    pick = np.where((dhi < dlo) | ((dhi == dlo) & odd), hi, lo)
    pick = np.where((b & np.uint32(0xFFFF)) == 0, b, pick)
    return (pick >> np.uint32(16)).astype(np.uint16)


def bf16_floats(h: np.ndarray) -> np.ndarray:
    """float32 values of bf16 bit patterns."""
    return (np.asarray(h).astype(np.uint32) << np.uint32(16)).view(np.float32)


def decode_slots(r) -> np.ndarray:
    """slots[leaf, row, 16 kh] (uint16) from the operand words, by the
    layout the header states: per leaf and k-half, rows in 32-point
    super-tiles of two 16-row m-tiles; row u's words sit at
    ((2 S + r) 8 + g) 16 + 2 a + 4 t + e (S = u / 32, a = u % 32 / 16,
    r = u % 16 / 8, g = u % 8), word (t, e) holding slots 2 (t + 4 e) and
    2 (t + 4 e) + 1 of the half.  Every word is written exactly once."""
    words, kh, stride = r["words"], r["kh"], r["stride"]
    L = len(r["leaf_lo"]) - 1
    u = np.arange(stride)
    S, a, rr, g = u // 32, (u % 32) // 16, (u % 16) // 8, u % 8
    slots = np.zeros((L, stride, 16 * kh), np.uint16)
    seen = np.zeros(words.size, np.int64)
    for leaf in range(L):
        for h in range(kh):
            base = ((leaf * kh + h) * stride * 8
                    + ((S * 2 + rr) * 8 + g) * 16 + 2 * a)
            for t in range(4):
                for e in range(2):
                    idx = base + 4 * t + e
                    w = words[idx]
                    k0 = 16 * h + 2 * (t + 4 * e)
                    slots[leaf, :, k0] = (w & 0xFFFF).astype(np.uint16)
                    slots[leaf, :, k0 + 1] = (w >> 16).astype(np.uint16)
                    np.add.at(seen, idx, 1)
    assert (seen == 1).all(), "operand words overlap or are left out"
    return slots


def decode_tc_slots(r) -> np.ndarray:
    """slots[leaf, row, 16 tc_kh] of the tcgen05 kernel's tiles, by the
    layout the header states (the MMA's no-swizzle K-major form): row r's
    slots 8 g .. 8 g + 7 at byte (r / 8) 256 kh + 128 g + 16 (r % 8) of its
    128-row tile.  Every element is written exactly once."""
    kh, tiles = r["tc_kh"], r["tiles"]
    L = len(r["leaf_lo"]) - 1
    words = r["tc_words"]
    tile_elems = 128 * 16 * kh
    rows = np.arange(128)
    slots = np.zeros((L, tiles * 128, 16 * kh), np.uint16)
    seen = np.zeros(words.size, np.int64)
    for leaf in range(L):
        for t in range(tiles):
            base = (leaf * tiles + t) * tile_elems
            for g in range(2 * kh):
                off = ((rows >> 3) * (256 * kh) + 128 * g + 16 * (rows & 7)) // 2
                for e in range(8):
                    idx = base + off + e
                    slots[leaf, t * 128 + rows, 8 * g + e] = words[idx]
                    np.add.at(seen, idx, 1)
    assert (seen == 1).all(), "tile elements overlap or are left out"
    return slots


def check_host_half(P: np.ndarray, h: int):
    """Every property of bkd_test_host_screen's output; returns the largest
    ||w - w_hat||^2 / max ||w_hat||^2 over the points of a leaf (exact): the
    rounding error a per-leaf bound from the leaf's largest operand norm
    must cover."""
    n, d = P.shape
    r = bkd.bkd_test_host_screen(P, h)
    L = 1 << h
    leaf_lo, perm = r["leaf_lo"], r["perm"]

    # the tree: the oracle's (same rule, independent code)
    ot = oracle.build_tree(P, h)
    assert np.array_equal(leaf_lo, ot.leaf_lo)
    assert np.array_equal(r["split"], ot.split[:L - 1])
    sizes = np.diff(leaf_lo)
    mine = np.empty(n, np.int64)
    mine[perm] = np.repeat(np.arange(L), sizes)
    assert np.array_equal(mine, ot.leaf_of_point())
    assert r["lcap"] == (sizes.max() + 3) // 4 * 4
    assert r["stride"] == (r["lcap"] + 31) // 32 * 32

    # node boxes: min / max of the points below, padding dimensions [0, 0]
    Dp, box = r["Dp"], r["box"]
    for v in range(2 * L - 1):
        lev = int(np.floor(np.log2(v + 1)))
        first = ((v + 1) << (h - lev)) - 1 - (L - 1)   # its leftmost leaf
        last = first + (1 << (h - lev))
        rows = P[perm[leaf_lo[first]:leaf_lo[last]]]
        assert np.array_equal(box[v, :d], rows.min(0)), v
        assert np.array_equal(box[v, Dp:Dp + d], rows.max(0)), v
        assert not box[v, d:Dp].any() and not box[v, Dp + d:].any()

    slots = decode_slots(r)
    # the tcgen05 kernel's rows: the same offsets and norm split, then three
    # 1.0 slots that meet the query's threshold parts; padding rows +inf
    tc = decode_tc_slots(r)
    for leaf in range(L):
        cnt = leaf_lo[leaf + 1] - leaf_lo[leaf]
        assert np.array_equal(tc[leaf, :cnt, :d + 2], slots[leaf, :cnt, :d + 2])
        assert (tc[leaf, :cnt, d + 2:d + 5] == 0x3F80).all()
        assert not tc[leaf, :cnt, d + 5:].any()
        assert (tc[leaf, cnt:, d] == 0x7F80).all()
        assert not np.delete(tc[leaf, cnt:], d, axis=1).any()
    half = np.float32(0.5)
    worst = Fraction(0)
    for leaf in range(L):
        rows = P[perm[leaf_lo[leaf]:leaf_lo[leaf + 1]]]
        cnt = rows.shape[0]
        c = r["center"][leaf]
        assert np.array_equal(c, half * rows.min(0) + half * rows.max(0))
        w32 = (rows - c).astype(np.float32)            # float32 subtraction
        wh = slots[leaf, :cnt, :d]
        assert np.array_equal(wh, bf16_nearest_even(w32)), leaf
        assert not slots[leaf, :cnt, d + 2:].any()
        pad = slots[leaf, cnt:]
        assert (pad[:, d] == 0x7F80).all()             # +inf norm
        assert not np.delete(pad, d, axis=1).any()
        bmax2 = Fraction(float(r["bmax"][leaf])) ** 2
        pnmax = Fraction(float(r["pnmax"][leaf]))
        # E >= 2^-14 pn_max >= 2^-100 covers every absolute (underflow) error
        # of the screen's arithmetic, all below 2^-118
        assert TWO ** -14 * pnmax >= TWO ** -100
        cf = [Fraction(float(x)) for x in c]
        whf = bf16_floats(wh)
        normf = bf16_floats(slots[leaf, :cnt, d:d + 2])
        wmax2 = Fraction(0)
        err2max = Fraction(0)
        for u in range(cnt):
            what = [Fraction(float(x)) for x in whf[u]]
            wtrue = [Fraction(float(x)) - ci for x, ci in zip(rows[u], cf)]
            err2 = sum((a - b) ** 2 for a, b in zip(wtrue, what))
            pn = sum(b * b for b in what)
            # the screen's bound: ||w - w_hat|| <= bmax of the leaf
            assert err2 <= bmax2, (leaf, u)
            assert pn <= pnmax, (leaf, u)
            # the norm split: relative error of the float32 sum and the two
            # bf16 parts, plus an absolute term once pn is subnormal (bf16
            # spacing there is 2^-133)
            parts = Fraction(float(normf[u, 0])) + Fraction(float(normf[u, 1]))
            assert abs(parts - pn) <= (TWO ** -16 + TWO ** -23) * pn \
                + TWO ** -133, (leaf, u)
            wmax2 = max(wmax2, pn)
            err2max = max(err2max, err2)
        if wmax2 > 0:
            worst = max(worst, err2max / wmax2)
    return worst


def near_tie_points(d: int, rng) -> np.ndarray:
    """One leaf (height 0) centred exactly on 1: two anchor rows 1 + D and
    1 - D in every dimension, D = (1 + 2^-8 - 2^-14) / 2 just below a bf16
    rounding tie (so the rows of largest operand norm carry a rounding error
    of almost 2^-8 of it); the other rows sit at 1 + delta, |delta| < D,
    with delta just below, at and just above ties over many exponents and
    both signs, mixed inside each row."""
    D = (1 + 2.0 ** -8 - 2.0 ** -14) / 2
    deltas = []
    for e in range(-2, -15, -1):
        for m in (1 + 2.0 ** -8 - 2.0 ** -14, 1 + 2.0 ** -8,
                  1 + 3 * 2.0 ** -8, 1 + 2.0 ** -8 + 2.0 ** -14,
                  1 + 2.0 ** -7 - 2.0 ** -15):
            for s in (1.0, -1.0):
                deltas.append(s * m * 2.0 ** e)
    deltas = np.array(deltas)
    rows = [np.full(d, 1.0 + D), np.full(d, 1.0 - D)]
    for _ in range(600):
        rows.append(1.0 + rng.choice(deltas, size=d))
    P = np.array(rows, np.float32)
    assert (P.astype(np.float64)[:2] == np.array(rows[:2])).all()
    return P


def test_host_tree_boxes_and_screen_operands_on_mixtures():
    for d, h, n in ((10, 4, 3000), (17, 3, 1500), (32, 2, 800), (3, 0, 50)):
        params = workloads.mixture_params(d, 8, 0.02, 0.2, d)
        P = workloads.mixture(n, params, 1 + d)
        check_host_half(P, h)


def test_screen_bound_holds_at_bf16_rounding_ties():
    rng = np.random.default_rng(20151209)
    worst = check_host_half(near_tie_points(10, rng), 0)
    # some point's error exceeds what a bound built on a 2^-9 rounding error
    # (2^-9 / (1 - 2^-9) times the leaf's largest operand norm) allows, so
    # such a bound would have failed above
    rho9 = TWO ** -9
    assert worst > (rho9 / (1 - rho9)) ** 2, float(worst)
    worst = check_host_half(near_tie_points(32, rng), 0)
    assert worst > (rho9 / (1 - rho9)) ** 2


@pytest.mark.parametrize("case", ["offset", "tiny", "subnormal", "dups"])
def test_screen_bound_on_hard_scales(case):
    rng = np.random.default_rng(7)
    if case == "offset":      # large common offset: x - c rounds in float32
        P = (rng.random((1200, 10)) + 1000.0).astype(np.float32)
    elif case == "tiny":      # leaves of spread 1e-4 around 0.3
        P = (0.3 + 1e-4 * rng.random((1200, 10))).astype(np.float32)
    elif case == "subnormal":  # float32 subnormals (below 2^-126)
        P = (rng.random((600, 6)) * 1e-39).astype(np.float32)
    else:                     # exact duplicates and a constant dimension
        base = rng.random((200, 5)).astype(np.float32)
        P = np.concatenate([base, base, base[:100]])
        P[:, 2] = 0.25
    check_host_half(P, 3)


def test_host_half_rejects_bad_arguments():
    P = np.zeros((10, 3), np.float32)
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_test_host_screen(P, 5)     # 32 leaves > 10 points
    assert e.value.code == bkd.BKD_EINVAL
    P[3, 1] = np.inf
    with pytest.raises(bkd.BkdError) as e:
        bkd.bkd_test_host_screen(P, 1)
    assert e.value.code == bkd.BKD_EINVAL
