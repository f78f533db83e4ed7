"""The two-float final merge of pass 2, checked against exact rationals.

Pass 2 ends every cohesion entry with error-free FP32 transformations
instead of FP64 instructions (cohesion_core.cuh: two_sum, inverse_pair,
mul_pair, cohesion_value, and the Fast2Sum fold of the running sums).  The
claim is that the merged value is the exact ((H - B) + S) / (n - 1) rounded
once to FP32, except when that exact value lies within 2^-46 of a rounding
midpoint (relative), where either neighbour may come out.

Here the same sequence of FP32 operations is restated in Python with every
operation done exactly in rationals and then rounded to nearest-even FP32
(an FMA rounds once), and compared with the exact quotient on 20,000 seeded
cases shaped like the kernel's operands.  A planted mistake (the low part of
1/(n-1) dropped) must fail, so the check has teeth.
"""
from fractions import Fraction as F

import numpy as np
import pytest

TWO = F(2)


def rn32(x: F) -> F:
    """x rounded to the nearest FP32 value, ties to even (normal range only)."""
    if x == 0:
        return F(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if a < TWO ** e:
        e -= 1
    assert TWO ** e <= a < TWO ** (e + 1)
    assert -126 <= e <= 127, "outside the normal FP32 range"
    m = a / TWO ** (e - 23)           # in [2^23, 2^24)
    q = m.numerator // m.denominator
    r = m - q
    if r > F(1, 2) or (r == F(1, 2) and q % 2 == 1):
        q += 1
    return sign * q * TWO ** (e - 23)


def f32(v) -> F:
    """An FP32 number (numpy float32 or Python value that is one) as a rational."""
    x = F(float(np.float32(v)))
    assert rn32(x) == x
    return x


# the FP32 operations the kernel uses, each rounded once
def fadd(a, b): return rn32(a + b)
def fsub(a, b): return rn32(a - b)
def fmul(a, b): return rn32(a * b)
def fma(a, b, c): return rn32(a * b + c)
def frcp(m): return rn32(1 / m)


# restatement of the kernel's merge steps
def two_sum(a, b):
    s = fadd(a, b)
    bv = fsub(s, a)
    e = fadd(fsub(a, fsub(s, bv)), fsub(b, bv))
    return s, e


def inverse_pair(m, drop_lo=False):
    mf = F(m)
    hi = frcp(mf)
    lo = fmul(fma(-hi, mf, F(1)), hi)
    return hi, (F(0) if drop_lo else lo)


def mul_pair(a, b, ih, il):
    m = fmul(a, ih)
    t = fma(a, ih, -m)
    return fadd(m, fma(a, il, fma(b, ih, t)))


def fast2sum_fold(h, s):
    t = fadd(h, s)
    z = fsub(t, h)
    return t, fsub(s, z)


BIAS = F(8)  # the running sums start at the bias kMergeBias = kMergeEvery = 8


def cohesion_value(H, S, n, drop_lo=False):
    ih, il = inverse_pair(n - 1, drop_lo)
    p, e = two_sum(fsub(H, BIAS), S)
    return mul_pair(p, e, ih, il)


def neighbours_ok(got, exact):
    """got == RN(exact), or exact is within 2^-46 (relative) of a midpoint
    and got is one of the two FP32 values around it."""
    want = rn32(exact)
    if got == want:
        return True
    lo, hi = sorted((got, want))
    mid = (lo + hi) / 2
    return abs(exact - mid) <= abs(exact) * TWO ** -46 and abs(got - want) <= abs(want) * TWO ** -22


def _cases(count, seed):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        n = int(rng.integers(2, 1 << 20))
        # running sum H = B + (a sum of up to n/2 terms of size <= 1/2): grid
        # of FP32 values of every magnitude the kernel can reach
        top = 8.0 + n / 2.0
        H = f32(8.0 + (top - 8.0) * rng.random() ** 3)
        # partial S: a few terms of 1/u, possibly a small negative carry
        S = f32(rng.random() * 4.0 - 1e-7 * rng.random())
        yield n, H, S


def test_inverse_pair_is_one_over_m_to_2_pow_minus_46():
    rng = np.random.default_rng(1)
    for m in list(range(1, 200)) + [int(v) for v in rng.integers(1, 1 << 24, size=2000)]:
        hi, lo = inverse_pair(m)
        assert abs(hi + lo - F(1, m)) <= F(1, m) * TWO ** -46


def test_fast2sum_fold_is_error_free_with_the_bias():
    rng = np.random.default_rng(2)
    for _ in range(5000):
        h = f32(8.0 + rng.random() * 1e5)
        s = f32(rng.random() * 4.0 - 1e-7)  # a partial over 8 y of terms <= 1/2
        assert abs(h) >= abs(s)
        t, e = fast2sum_fold(h, s)
        assert t + e == h + s


def test_merge_is_correctly_rounded_on_20000_cases():
    bad = []
    for n, H, S in _cases(20000, seed=3):
        got = cohesion_value(H, S, n)
        exact = ((H - BIAS) + S) / (n - 1)
        if exact == 0:
            assert got == 0
            continue
        if not neighbours_ok(got, exact):
            bad.append((n, float(H), float(S)))
    assert not bad, f"{len(bad)} cases not correctly rounded, e.g. {bad[:3]}"


def test_planted_mistake_is_caught():
    # dropping the low part of 1/(n-1) leaves an error of up to 2^-24
    # relative before the final rounding: some case must then round wrongly
    caught = 0
    for n, H, S in _cases(4000, seed=4):
        exact = ((H - BIAS) + S) / (n - 1)
        if exact != 0 and not neighbours_ok(cohesion_value(H, S, n, drop_lo=True), exact):
            caught += 1
    assert caught > 0


@pytest.mark.parametrize("m", [1, 2, 3, 5, 7, 65535, (1 << 20) - 1])
def test_exact_small_quotients(m):
    # H - B + S equal to a multiple of (n - 1): the result must be exact
    n = m + 1
    for k in (1, 3, 17):
        if 8 + k * m >= 1 << 24:  # H must be an FP32 integer (it never exceeds 8 + n/2)
            continue
        H = f32(8.0 + k * m)
        got = cohesion_value(H, F(0), n)
        assert got == k
