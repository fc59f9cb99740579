"""Pins of the oracle's binary32 conversion against what the formats and the
mathematics fix (Section 2: binary32 has a 24-bit significand, normal
exponents -126..127, subnormals down to 2^-149):

* round trips: 9 significant digits (and numpy's shortest repr) of any
  float32 parse back to that float32;
* constructed midpoints between adjacent float32 values, written out in
  full: a tie goes to the even significand, one unit more or less in the
  last digit goes to that side;
* exact integers (all of [0, 2^24] exact; above, the closed-form
  round-half-even to the grid) and exact powers of ten (10^k exact for
  k <= 10, since 5^10 < 2^24 < 5^11);
* range boundaries (2^-150 ties to 0, above it 2^-149; the overflow
  threshold (2^24 - 1/2) 2^104);
* brute force: every 1-3 digit significand times 10^E, E in [-50, 40],
  against the nearest of the candidate's neighbours by exact rational
  comparison (a different method from the oracle's long division).
"""
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle

OK, INVALID, OVERFLOW, UNDERFLOW = 0, 1, 2, 3
INF32 = 0x7F800000


def f32_value(bits: int) -> Fraction:
    """Exact value of a positive finite binary32 pattern."""
    e, m = bits >> 23, bits & 0x7FFFFF
    if e == 0:
        return Fraction(m, 2 ** 149)
    return Fraction(m | 0x800000) * Fraction(2) ** (e - 150)


def exact_decimal(v: Fraction) -> str:
    """The exact decimal expansion of a dyadic rational (denominator 2^k)."""
    num, den = v.numerator, v.denominator
    k = den.bit_length() - 1
    assert den == 1 << k
    return "%de-%d" % (num * 5 ** k, k) if k else str(num)


def bump_last_digit(s: str, delta: int) -> str:
    """s = digits 'e-' k: add delta to the integer of digits."""
    digits, _, k = s.partition("e-")
    return "%de-%s" % (int(digits) + delta, k) if k else str(int(digits) + delta)


def nearest_f32(v: Fraction) -> int:
    """Nearest positive binary32 pattern to v >= 0 by comparing v with the
    exact values of a candidate and its neighbours (ties to even)."""
    if v == 0:
        return 0
    overflow_at = (Fraction(2 ** 24) - Fraction(1, 2)) * Fraction(2) ** 104
    if v >= overflow_at:
        return INF32  # at or beyond the midpoint of FLT_MAX and 2^128 (FLT_MAX is odd)
    c = int(np.array([float(v)], dtype=np.float64).astype(np.float32).view(np.uint32)[0])
    cands = [b for b in (c - 1, c, c + 1) if 0 <= b < INF32]
    best = min(cands, key=lambda b: (abs(f32_value(b) - v), b & 1))
    # neither neighbour of the best may be closer
    for b in (best - 1, best + 1):
        if 0 <= b < INF32:
            assert abs(f32_value(b) - v) >= abs(f32_value(best) - v)
    return best


def parse32(s):
    return oracle.parse_field_f32(s)


def random_finite_f32(rnd, count, subnormal_share=0.1):
    out = []
    for _ in range(count):
        if rnd.random() < subnormal_share:
            out.append(rnd.randrange(1, 1 << 23))
        else:
            out.append(rnd.randrange(1 << 23, INF32))
    return out


def test_nine_digit_round_trip():
    rnd = random.Random(1)
    for b in random_finite_f32(rnd, 30000):
        x = float(np.array([b], dtype=np.uint32).view(np.float32)[0])
        for s in ("%.9g" % x, "%.9e" % -x):
            got, st = parse32(s)
            want = b | (0x80000000 if s.startswith("-") else 0)
            assert (got, st) == (want, OK), s


def test_shortest_repr_round_trip():
    rnd = random.Random(2)
    for b in random_finite_f32(rnd, 20000):
        x = np.array([b], dtype=np.uint32).view(np.float32)[0]
        for s in (np.format_float_scientific(x, unique=True),
                  np.format_float_positional(x, unique=True)):
            assert parse32(s) == (b, OK), s


def test_constructed_midpoints():
    rnd = random.Random(3)
    bits = random_finite_f32(rnd, 3000, subnormal_share=0.3) + [1, 2, 0x7FFFFF, 0x800000,
                                                               0x7F7FFFFE]
    for b in bits:
        lo, hi = f32_value(b), f32_value(b + 1)
        mid = (lo + hi) / 2
        s = exact_decimal(mid)
        even = b if b % 2 == 0 else b + 1
        assert parse32(s) == (even, OK), s
        assert parse32(bump_last_digit(s, +1)) == (b + 1, OK)
        assert parse32(bump_last_digit(s, -1)) == (b, OK)
    # between FLT_MAX (odd) and 2^128: the tie goes to infinity
    mid = (f32_value(0x7F7FFFFF) + Fraction(2) ** 128) / 2
    assert parse32(exact_decimal(mid)) == (INF32, OVERFLOW)
    assert parse32(bump_last_digit(exact_decimal(mid), -1)) == (0x7F7FFFFF, OK)


def test_exact_integers_and_their_rounding():
    rnd = random.Random(4)
    ns = list(range(0, 5000)) + [rnd.randrange(0, 1 << 24) for _ in range(5000)] + [1 << 24]
    for n in ns:
        want = int(np.array([n], dtype=np.float32).view(np.uint32)[0])  # exact: n <= 2^24
        assert f32_value(want) == n
        assert parse32(str(n)) == (want, OK)
    # [2^24, 2^25): the grid step is 2; half-way integers go to the even multiple
    for n in [(1 << 24) + k for k in range(0, 64)] + [rnd.randrange(1 << 24, 1 << 25)
                                                       for _ in range(2000)]:
        q, r = divmod(n, 2)
        if r == 1 and q % 2 == 1:
            q += 1
        got, st = parse32(str(n))
        assert st == OK and f32_value(got) == 2 * q, n


def test_powers_of_ten():
    for k in range(0, 11):
        got, st = parse32("1e%d" % k)
        assert st == OK and f32_value(got) == 10 ** k
    got, _ = parse32("1e11")
    assert f32_value(got) != 10 ** 11          # 5^11 > 2^24: not exact
    assert got == nearest_f32(Fraction(10) ** 11)
    for k in range(-45, 39):
        assert parse32("1e%d" % k)[0] == nearest_f32(Fraction(10) ** k), k


def test_range_boundaries():
    tiny = Fraction(1, 2 ** 149)
    assert parse32(exact_decimal(tiny / 2)) == (0, UNDERFLOW)          # tie with 0: even
    assert parse32(bump_last_digit(exact_decimal(tiny / 2), 1)) == (1, OK)
    assert parse32(exact_decimal(tiny * 3 / 2)) == (2, OK)             # tie between 1 and 2
    assert parse32(exact_decimal(tiny)) == (1, OK)
    assert parse32("1e-46") == (0, UNDERFLOW)
    assert parse32("-1e-46") == (0x80000000, UNDERFLOW)
    assert parse32(exact_decimal(Fraction(1, 2 ** 126))) == (0x800000, OK)
    assert parse32("3.4028235e38") == (0x7F7FFFFF, OK)
    assert parse32("3.4028236e38") == (INF32, OVERFLOW)
    assert parse32("-1e39") == (INF32 | 0x80000000, OVERFLOW)
    assert parse32("0e999") == (0, OK) and parse32("-0.0") == (0x80000000, OK)
    assert parse32("1e") == (0x7FC00000, INVALID)


def test_brute_force_small_significands():
    for E in range(-50, 41):
        for d in list(range(1, 1000, 7)) + [1, 9, 99, 999]:
            s = "%de%d" % (d, E)
            want = nearest_f32(Fraction(d) * Fraction(10) ** E)
            got, st = parse32(s)
            assert got == want, s
            assert st == (OVERFLOW if want == INF32 else UNDERFLOW if want == 0 else OK)


def test_long_significands():
    """More digits than any fast path keeps: a midpoint written with
    hundreds of trailing zeros, and a nonzero digit far out."""
    rnd = random.Random(5)
    for b in random_finite_f32(rnd, 200, subnormal_share=0.5):
        mid = (f32_value(b) + f32_value(b + 1)) / 2
        digits, _, k = exact_decimal(mid).partition("e-")
        k = int(k or 0)
        s = digits + "0" * 300 + "e-%d" % (k + 300)
        even = b if b % 2 == 0 else b + 1
        assert parse32(s) == (even, OK)
        assert parse32(digits + "0" * 300 + "1e-%d" % (k + 301)) == (b + 1, OK)


def test_buffer_form_matches_fields():
    fields = ["1.5", "-2e-40", "", "3.4e38", "x", "1e39", "0.1", "16777217"]
    text = "\n".join(fields).encode()
    bits, st = oracle.parse_buffer(text, f32=True)
    assert bits.dtype == np.uint32 and bits.size == len(fields)
    for i, f in enumerate(fields):
        assert (int(bits[i]), int(st[i])) == parse32(f)
