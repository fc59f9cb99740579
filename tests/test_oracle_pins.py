"""Pins for the CPU oracle against facts fixed outside the oracle itself.

Each test ties the oracle to something it cannot satisfy by construction:
values the paper prints, closed forms (exact integers, exact powers of ten,
midpoints between adjacent doubles built with exact integer arithmetic),
and CPython's float(), which is a correctly rounded decimal-to-binary64
library routine.  The oracle never calls float() on a decimal string.
"""
import math
import os
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2101_11408_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DBL_MAX_BITS = 0x7FEFFFFFFFFFFFFF
INF_BITS = 0x7FF0000000000000


def f2b(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def exact_bits(value: Fraction) -> int:
    """Bits of a binary64 that equals `value` exactly (asserted)."""
    x = float(value)  # Fraction -> float is correctly rounded
    assert Fraction(x) == value, "expected value is not a binary64"
    return f2b(x)


def parse(s):
    return oracle.parse_field(s)


def parse_many(strings, delim=b"\n"):
    text = "\n".join(strings).encode("latin-1")
    bits, st = oracle.parse_buffer(text, delim)
    assert bits.size == len(strings)
    return bits, st


# --------------------------------------------------------------------------
# values printed in the paper
# --------------------------------------------------------------------------

def _golden_examples():
    rows = []
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            inp, exp, where = line.rstrip("\n").split("\t")
            rows.append((inp, exp, where))
    return rows


@pytest.mark.parametrize("inp,expected,where", _golden_examples())
def test_paper_worked_examples(inp, expected, where):
    bits, st = parse(inp)
    assert st == oracle.STATUS_OK
    if expected.startswith("0x"):
        assert bits == f2b(float.fromhex(expected)), where
    elif expected.startswith("sig="):
        m = int(expected[4:])
        # the significand the paper prints, and the binade of the exact value:
        # floor(log2 V) computed from integer bit lengths
        w, q = inp.split("e")
        V = Fraction(int(w)) * Fraction(10) ** int(q)
        k = V.numerator.bit_length() - V.denominator.bit_length()
        if Fraction(2) ** k > V:
            k -= 1
        assert (bits & ((1 << 52) - 1)) | (1 << 52) == m, where
        assert (bits >> 52) - 1023 == k, where
    else:
        M, E = expected.split("*2^")
        assert bits == exact_bits(Fraction(int(M)) * Fraction(2) ** int(E)), where


def test_768_digit_midpoint_rounds_up():
    """Section 11: 2^-1022 + 2^-1074 + 2^-1075 needs 768 significant digits and
    is a tie that rounds to the even neighbour 2^-1022 + 2^-1073."""
    V = Fraction(2) ** -1022 + Fraction(2) ** -1074 + Fraction(2) ** -1075
    n = V.numerator * 5 ** 1075  # V = n / 10^1075 exactly
    assert V.denominator == 2 ** 1075
    digits = str(n).rstrip("0")
    assert len(digits) == 768
    s = "0." + "0" * (1075 - len(str(n))) + str(n)
    bits, st = parse(s)
    assert st == oracle.STATUS_OK
    assert bits == f2b(float.fromhex("0x1.0000000000002p-1022"))
    # one unit lower in the last place rounds down instead
    lower = str(n - 10 ** (len(str(n)) - len(digits)))
    s2 = "0." + "0" * (1075 - len(lower)) + lower
    assert parse(s2)[0] == f2b(float.fromhex("0x1.0000000000001p-1022"))


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_exact_integers_up_to_2_53():
    rnd = random.Random(11)
    vals = [0, 1, 2, 9, 10, 2 ** 52 - 1, 2 ** 52, 2 ** 52 + 1, 2 ** 53 - 1, 2 ** 53]
    vals += [rnd.randrange(0, 2 ** 53 + 1) for _ in range(20000)]
    vals += [rnd.randrange(0, 10 ** rnd.randrange(1, 16)) for _ in range(20000)]
    bits, st = parse_many([str(v) for v in vals])
    assert (st == 0).all()
    for v, b in zip(vals, bits.tolist()):
        assert b == exact_bits(Fraction(v))


def test_exact_powers_of_ten():
    """Section 6: 10^q is exact in binary64 for q in [0, 22], not for 23."""
    for k in range(0, 23):
        for s in ("1e%d" % k, "1" + "0" * k, "0.1e%d" % (k + 1)):
            b, st = parse(s)
            assert st == 0 and b == exact_bits(Fraction(10) ** k)
    b, _ = parse("1e23")
    x = struct.unpack("<d", struct.pack("<Q", b))[0]
    assert Fraction(x) != Fraction(10) ** 23


def test_roundtrip_17_digits():
    """Section 1: 17 significant digits always parse back to the same double."""
    rng = np.random.Generator(np.random.PCG64(7))
    raw = rng.integers(0, 2 ** 63 - 1, size=60000, dtype=np.int64)
    xs = raw.view(np.float64)
    xs = xs[np.isfinite(xs)]
    strs = ["%.17g" % x for x in xs.tolist()] + [repr(-x) for x in xs[:20000].tolist()]
    want = [f2b(x) for x in xs.tolist()] + [f2b(-x) for x in xs[:20000].tolist()]
    bits, st = parse_many(strs)
    assert (st == 0).all()
    assert bits.tolist() == want


def _midpoint_cases(bits_list):
    strs, want = [], []
    for b in bits_list:
        digits, e10 = workloads.midpoint_decimal(b)
        lo, hi = b, b + 1
        even = lo if (lo & 1) == 0 else hi
        for delta, exp in ((0, even), (1, hi), (-1, lo)):
            d = str(int(digits) + delta)
            strs.append("%se%d" % (d, e10))
            want.append(exp)
    return strs, want


def test_constructed_midpoints():
    """Exact midpoints between adjacent doubles: ties go to the even
    significand; one unit up or down in the last digit decides the side."""
    rng = np.random.Generator(np.random.PCG64(3))
    normal = rng.integers(0x0010000000000000, DBL_MAX_BITS, size=1500, dtype=np.int64)
    sub = rng.integers(0, 0x0010000000000000, size=600, dtype=np.int64)
    edges = [0, 1, 2, 0x000FFFFFFFFFFFFF, 0x0010000000000000, 0x3FEFFFFFFFFFFFFF,
             0x3FF0000000000000, 0x433FFFFFFFFFFFFF, 0x4340000000000000, DBL_MAX_BITS - 1,
             DBL_MAX_BITS]
    strs, want = _midpoint_cases([int(b) for b in normal] + [int(b) for b in sub] + edges)
    bits, st = parse_many(strs)
    for s, b, w, t in zip(strs, bits.tolist(), want, st.tolist()):
        assert b == w, s[:60]
        if w == INF_BITS:
            assert t == oracle.STATUS_OVERFLOW
        elif w == 0:
            assert t == oracle.STATUS_UNDERFLOW
        else:
            assert t == oracle.STATUS_OK


def test_range_boundaries():
    half_min = Fraction(2) ** -1075
    n = half_min.numerator * 5 ** 1075
    s = "0." + "0" * (1075 - len(str(n))) + str(n)
    assert parse(s) == (0, oracle.STATUS_UNDERFLOW)          # tie -> even 0
    assert parse(s + "1") == (1, oracle.STATUS_OK)           # just above
    assert parse("-" + s + "1") == (1 | (1 << 63), oracle.STATUS_OK)
    assert parse("-" + s) == (1 << 63, oracle.STATUS_UNDERFLOW)
    digits, e10 = workloads.midpoint_decimal(DBL_MAX_BITS)   # DBL_MAX + half ulp
    assert parse("%se%d" % (digits, e10)) == (INF_BITS, oracle.STATUS_OVERFLOW)
    assert parse("%se%d" % (str(int(digits) - 1), e10)) == (DBL_MAX_BITS, oracle.STATUS_OK)
    assert parse("1e309") == (INF_BITS, oracle.STATUS_OVERFLOW)
    assert parse("-1e309") == (INF_BITS | (1 << 63), oracle.STATUS_OVERFLOW)
    assert parse("1e-400") == (0, oracle.STATUS_UNDERFLOW)
    assert parse("0e999999999999") == (0, oracle.STATUS_OK)
    assert parse("-0.000") == (1 << 63, oracle.STATUS_OK)


# --------------------------------------------------------------------------
# CPython's correctly rounded float() as the library routine
# --------------------------------------------------------------------------

def _random_strings(rnd: random.Random, n: int):
    out = []
    for _ in range(n):
        kind = rnd.randrange(8)
        nd = rnd.randrange(1, 40) if kind < 6 else rnd.randrange(40, 120)
        digs = "".join(rnd.choice("0123456789") for _ in range(nd))
        if kind == 0:
            s = digs
        elif kind == 1:
            p = rnd.randrange(0, nd + 1)
            s = digs[:p] + "." + digs[p:]
        elif kind in (2, 6):
            s = digs + "e" + str(rnd.randrange(-360, 330))
        elif kind in (3, 7):
            p = rnd.randrange(0, nd + 1)
            s = digs[:p] + "." + digs[p:] + rnd.choice("eE") + rnd.choice(["", "+", "-"]) + \
                str(rnd.randrange(0, 340))
        elif kind == 4:  # subnormal range
            s = "%se-%d" % (digs, rnd.randrange(300, 345) + nd)
        else:  # near overflow
            s = "%se%d" % (digs, 308 - nd + rnd.randrange(-2, 3))
        if s.startswith("."):
            s = "0" + s if rnd.random() < 0.5 else s
        if s.endswith(".") or s.startswith("."):
            pass
        if s == "." or s.startswith(".e") or s.startswith(".E"):
            s = "0" + s
        if rnd.random() < 0.3:
            s = rnd.choice("+-") + s
        out.append(s)
    return out


def test_random_strings_match_cpython_float():
    rnd = random.Random(2101)
    strs = _random_strings(rnd, 150000)
    bits, st = parse_many(strs)
    for s, b in zip(strs, bits.tolist()):
        assert b == f2b(float(s)), s


def test_small_significands_all_exponents():
    """Every 1..3 digit significand times 10^E for E in [-345, 310]."""
    strs = ["%de%d" % (m, e) for m in range(1, 1000) for e in range(-345, 311)]
    bits, st = parse_many(strs)
    want = np.array([f2b(float(s)) for s in strs], dtype=np.uint64)
    assert np.array_equal(bits, want)
    inf = want == INF_BITS
    zero = want == 0
    assert (st[inf] == oracle.STATUS_OVERFLOW).all()
    assert (st[zero] == oracle.STATUS_UNDERFLOW).all()
    assert (st[~inf & ~zero] == oracle.STATUS_OK).all()


def test_long_significands_match_cpython_float():
    rnd = random.Random(5)
    strs = []
    for _ in range(3000):
        nd = rnd.randrange(20, 900)
        d = rnd.choice("123456789") + "".join(rnd.choice("0123456789") for _ in range(nd - 1))
        p = rnd.randrange(1, nd)
        strs.append("%s.%se%d" % (d[:p], d[p:], rnd.randrange(-330, 300) - p))
    bits, _ = parse_many(strs)
    for s, b in zip(strs, bits.tolist()):
        assert b == f2b(float(s))


def test_bulk_workload_matches_cpython_float():
    lines = workloads.bulk_mixed_lines(40000, 99)
    bits, _ = parse_many(lines)
    assert bits.tolist() == [f2b(float(s)) for s in lines]


# --------------------------------------------------------------------------
# grammar, statuses and buffer rules
# --------------------------------------------------------------------------

GRAMMAR = [
    ("1", True), ("+1", True), ("-1", True), ("1.", True), (".5", True), ("1.e1", True),
    ("1e+1", True), ("10E-01", True), (" \t1\r", True), ("  -0.5e-3 ", True),
    ("007", True), ("0.000", True),
    ("", False), (" ", False), (".", False), ("+", False), ("-", False), ("e5", False),
    (".e5", False), ("1e", False), ("1e+", False), ("1e-", False), ("+-1", False),
    ("--1", False), ("1..2", False), ("1.2.3", False), ("1e5.5", False), ("1 2", False),
    ("0x1p3", False), ("inf", False), ("nan", False), ("1,5", False), ("1e5e5", False),
    ("١", False), ("1\x00", False), ("1\v", False), ("1_000", False),
]


@pytest.mark.parametrize("s,valid", GRAMMAR)
def test_grammar(s, valid):
    bits, st = parse(s)
    if valid:
        assert st == oracle.STATUS_OK
        assert bits == f2b(float(s.strip(" \t\r")))
    else:
        assert st == oracle.STATUS_INVALID
        assert bits == 0x7FF8000000000000


def test_sign_of_zero_and_infinity():
    assert parse("-0") == (1 << 63, 0)
    assert parse("+0.0e5") == (0, 0)
    assert parse("-1e-400") == (1 << 63, oracle.STATUS_UNDERFLOW)
    assert parse("-1e400") == (INF_BITS | 1 << 63, oracle.STATUS_OVERFLOW)


def test_exponent_saturation_is_harmless():
    assert parse("1e99999999999999999999999") == (INF_BITS, oracle.STATUS_OVERFLOW)
    assert parse("1e-99999999999999999999999") == (0, oracle.STATUS_UNDERFLOW)
    assert parse("0." + "0" * 500 + "1e520")[0] == f2b(1e19)


def test_buffer_field_rules():
    cases = [
        (b"", b"\n", []),
        (b"1", b"\n", ["1"]),
        (b"1\n", b"\n", ["1"]),
        (b"1\n2", b"\n", ["1", "2"]),
        (b"1\n\n2\n", b"\n", ["1", "", "2"]),
        (b"\n", b"\n", [""]),
        (b"\n\n", b"\n", ["", ""]),
        (b"1,2\n3,", b",", ["1", "2", "3"]),
        (b"1,2\r\n3", b",", ["1", "2\r", "3"]),
    ]
    for text, delim, fields in cases:
        assert oracle.count_fields(text, delim) == len(fields)
        bits, st = oracle.parse_buffer(text, delim)
        assert bits.size == len(fields)
        for f, b, t in zip(fields, bits.tolist(), st.tolist()):
            assert (b, t) == parse(f)


def test_thread_count_does_not_change_results():
    text = workloads.bulk_mixed_text(60000, 17)
    b1, s1 = oracle.parse_buffer(text, b"\n", nthreads=1)
    b8, s8 = oracle.parse_buffer(text, b"\n", nthreads=8)
    assert np.array_equal(b1, b8) and np.array_equal(s1, s8)


def test_hard_case_workload_matches_cpython_float():
    lines = workloads.hard_case_lines(3000, 1234)
    bits, _ = parse_many(lines)
    for s, b in zip(lines, bits.tolist()):
        assert b == f2b(float(s)), s[:80]
