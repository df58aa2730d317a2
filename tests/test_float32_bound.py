"""The two facts about float32 arithmetic that make the GPU path exact, checked
on the CPU in exact rational arithmetic (no GPU, no library call):

1. Error bound of the float32 distance chain (the leaf, tail and screen
   rescoring kernels' t_i = fl(q_i - x_i), e = fl(t_0^2), e = fma(t_i, t_i, e)):
   |v - D64| <= gam D64 + eta with gam = (d + 3) 2^-24 and eta = 2^-120,
   D64 the oracle's binary64 distance.  The re-check classifies a query's
   list as final from intervals built on this bound (Sec. 2.2's exact
   answer), so the bound must hold on every input, including cancellation,
   huge and subnormal coordinates.
2. Exact pruning (the traversal's bounding-box test): the same chain over
   o_i = max(fl(lo_i - q_i), fl(q_i - hi_i), 0) is never above the chain of
   any point x inside the box [lo, hi], so skipping a subtree whose box bound
   reaches the list's bound never drops a point that would enter the list.

Float32 rounding is emulated from its definition (round to nearest, ties to
even, gradual underflow), checked against numpy's conversion first.  Planted
mistakes (one rounding per term in gam; the box chain with a separate
multiply and add) fail the checks.
"""
from fractions import Fraction

import numpy as np

U = Fraction(1, 1 << 24)
ETA = Fraction(1, 1 << 120)


def round_f32(x: Fraction) -> Fraction:
    """x rounded to the nearest float32 (ties to even, subnormals below
    2^-126); |x| stays far below the float32 overflow here."""
    if x == 0:
        return Fraction(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    quantum = Fraction(2) ** max(e - 23, -149)
    scaled = a / quantum
    n = scaled.numerator // scaled.denominator
    rest = scaled - n
    if rest > Fraction(1, 2) or (rest == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * n * quantum


def chain32(t):
    """fl(t_0^2), then fma(t_i, t_i, e): one rounding per operation."""
    e = round_f32(t[0] * t[0])
    for ti in t[1:]:
        e = round_f32(ti * ti + e)
    return e


def dist32(q, x):
    return chain32([round_f32(Fraction(float(a)) - Fraction(float(b)))
                    for a, b in zip(q, x)])


def dist64(q, x) -> Fraction:
    """The oracle's binary64 sequence (Python floats are IEEE binary64)."""
    acc = 0.0
    for a, b in zip(q, x):
        t = float(a) - float(b)
        acc = acc + t * t
    return Fraction(acc)


def box_bound32(q, lo, hi):
    o = []
    for qi, l, h in zip(q, lo, hi):
        qf, lf, hf = Fraction(float(qi)), Fraction(float(l)), Fraction(float(h))
        o.append(max(round_f32(lf - qf), round_f32(qf - hf), Fraction(0)))
    return chain32(o)


def test_round_f32_is_numpys_conversion():
    rng = np.random.default_rng(3)
    vals = np.concatenate([rng.standard_normal(4000),
                           rng.standard_normal(1000) * 1e-40,
                           rng.standard_normal(1000) * 1e30,
                           (1 + rng.integers(0, 1 << 29, 1000) * 2.0 ** -29),
                           np.array([1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24,
                                     2.0 ** -149 * 0.5, 2.0 ** -149 * 1.5,
                                     -(1 + 2.0 ** -24), 2.0 ** -126 * 0.75])])
    for v in vals:
        assert round_f32(Fraction(float(v))) == Fraction(float(np.float32(v)))


def cases(rng):
    """(q, x) float32 pairs: ordinary data, near-identical pairs (heavy
    cancellation), huge and subnormal coordinates, mixed scales."""
    out = []
    for d in (1, 2, 3, 10, 17, 32):
        for kind in range(6):
            for _ in range(12):
                if kind == 0:
                    q, x = rng.random(d), rng.random(d)
                elif kind == 1:
                    q = rng.random(d) * 100
                    x = q + rng.standard_normal(d) * 1e-5 * q
                elif kind == 2:
                    q, x = rng.standard_normal((2, d)) * 1e17
                elif kind == 3:
                    q, x = rng.standard_normal((2, d)) * 1e-39
                elif kind == 4:
                    scale = 10.0 ** rng.integers(-30, 30, d)
                    q, x = (rng.standard_normal((2, d)) * scale)
                else:
                    q = 1 + rng.integers(0, 1 << 20, d) * 2.0 ** -23
                    x = -(2.0 ** -24) * (1 - rng.random(d) * 2.0 ** -10)
                out.append((np.float32(q), np.float32(x)))
    return out


def test_float32_chain_error_bound():
    rng = np.random.default_rng(1512)
    worst = 0.0
    for q, x in cases(rng):
        d = q.size
        v, D64 = dist32(q, x), dist64(q, x)
        gam = (d + 3) * U
        assert abs(v - D64) <= gam * D64 + ETA, (q, x)
        if D64 > 2 ** -100:
            worst = max(worst, float(abs(v - D64) / D64 / U) / (d + 3))
    assert worst < 1.0


def test_a_bound_of_one_rounding_per_term_is_too_small():
    """d = 1, q - x just below a float32 rounding tie: the subtraction loses
    almost 2^-24 of t, the square doubles it, so gam = d 2^-24 (one rounding
    per term, the subtraction forgotten) is exceeded; (d + 3) 2^-24 is not."""
    q = np.float32([1.0])
    x = np.float32([-(2.0 ** -24) * (1 - 2.0 ** -16)])
    v, D64 = dist32(q, x), dist64(q, x)
    assert abs(v - D64) > 1 * U * D64
    assert abs(v - D64) <= 4 * U * D64


def test_box_bound_never_exceeds_a_point_inside():
    rng = np.random.default_rng(2)
    for d in (1, 2, 3, 10):
        for _ in range(150):
            a, b = rng.standard_normal((2, d)) * 10.0 ** rng.integers(-3, 4)
            lo, hi = np.float32(np.minimum(a, b)), np.float32(np.maximum(a, b))
            q = np.float32(rng.standard_normal(d) * 10.0 ** rng.integers(-3, 4))
            # points inside: corners (the tightest), face points, random
            pts = [np.where(rng.random(d) < 0.5, lo, hi),
                   np.float32(np.clip(q, lo, hi)),
                   np.float32(lo + (hi - lo) * rng.random(d))]
            B = box_bound32(q, lo, hi)
            for x in pts:
                x = np.float32(np.clip(x, lo, hi))
                assert B <= dist32(q, x), (q, lo, hi, x)


def test_a_box_chain_with_separate_multiply_and_add_can_exceed_a_point():
    """The box bound must use the points' own chain (fused multiply-add).
    With a separate multiply and add (two roundings) it can exceed the
    distance of the box's nearest point, which would prune a true
    neighbour: found here by search."""
    def chain_mul_add(t):
        e = round_f32(t[0] * t[0])
        for ti in t[1:]:
            e = round_f32(round_f32(ti * ti) + e)
        return e

    rng = np.random.default_rng(5)
    found = False
    for _ in range(3000):
        d = 3
        q = np.float32(rng.random(d))
        x = np.float32(q + rng.standard_normal(d) * 0.3)
        # a degenerate box holding only x: its bound is x's own o_i
        o = [max(round_f32(Fraction(float(xi)) - Fraction(float(qi))),
                 round_f32(Fraction(float(qi)) - Fraction(float(xi))),
                 Fraction(0)) for qi, xi in zip(q, x)]
        if chain_mul_add(o) > dist32(q, x):
            found = True
            break
    assert found
