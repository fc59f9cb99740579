"""The seeded synthetic workloads hold the recipes the measurements are
quoted on: deterministic in their seed, with the stated shapes and
proportions (bulk: 40% uniform %.17g, 30% coordinates, 20% integers below
2^63, 10% d.ddddE+-xxx; hard: long digit strings, exact midpoints, range
ends; batched sizes lognormal with sigma 2 summing to the total; hex floats
that are exact float.hex() images; 8-column CSV rows)."""
import math
import re

import numpy as np
import pytest

from paper_2101_11408_gb300 import workloads as w


@pytest.mark.parametrize("gen", [w.uniform_text, w.bulk_mixed_text, w.hard_case_text,
                                 w.hex_float_text])
def test_deterministic_in_the_seed(gen):
    a, b, c = gen(3000, 11), gen(3000, 11), gen(3000, 12)
    assert a == b and a != c
    assert a.count(b"\n") == 2999 and not a.endswith(b"\n")


def test_bulk_mix_shares_and_shapes():
    lines = w.bulk_mixed_lines(50000, 21)
    sci = [s for s in lines if "E" in s]
    ints = [s for s in lines if s.isdigit()]
    rest = [s for s in lines if "E" not in s and not s.isdigit()]
    uni = [s for s in rest if re.fullmatch(r"0\.\d+|\d\.\d+e-\d+", s) and float(s) < 1]
    uni_set = set(uni)
    coord = [s for s in rest if s not in uni_set]
    for got, share in ((uni, 0.4), (coord, 0.3), (ints, 0.2), (sci, 0.1)):
        assert abs(len(got) / len(lines) - share) < 0.01, (share, len(got))
    assert all(re.fullmatch(r"[1-9]\.\d{4}E[+-]\d{3}", s) for s in sci)
    assert all(-340 <= int(s[-4:]) <= 320 for s in sci)
    assert all(int(s) < 2 ** 63 for s in ints)
    fr = [len(s.split(".")[1]) for s in coord]
    assert min(fr) == 12 and max(fr) == 16
    assert all(abs(float(s)) <= 180 for s in coord)
    # the uniform values keep 17 significant digits (%.17g)
    assert np.mean([len(s.replace("0.", "", 1).lstrip("0").split("e")[0]) for s in uni]) > 16
    text = w.bulk_mixed_text(50000, 21)
    assert 18.0 < len(text) / 50000 < 19.6  # about 18.8 bytes per number


def test_hard_mix_shapes():
    lines = w.hard_case_lines(6000, 31)

    def sig_digits(s):
        m = s.lstrip("+-").split("e")[0].split("E")[0].replace(".", "").lstrip("0")
        return len(m.rstrip("0")) or 1
    long_ = [s for s in lines if sig_digits(s) >= 20]
    assert len(long_) / len(lines) > 0.5  # the 20-800 digit half, and many midpoints
    assert max(sig_digits(s) for s in lines) > 700


def test_batched_sizes():
    total, count = 2 << 30, 4096
    sizes = np.array(w.lognormal_sizes(count, total, 1 << 10, 64 << 20, 2.0, 41))
    assert sizes.min() >= 1 << 10 and sizes.max() <= 64 << 20
    assert abs(sizes.sum() / total - 1) < 0.01
    inner = np.log(sizes[(sizes > 1 << 10) & (sizes < 64 << 20)])
    assert 1.6 < inner.std() < 2.2  # sigma 2, narrowed by the clipping


def test_hex_floats_are_float_hex_images():
    lines = w.hex_float_lines(4000, 51)
    xs = [float.fromhex(s) for s in lines]
    assert all(x.hex() == s for x, s in zip(xs, lines))
    unit = sum(1 for x in xs if 0 <= x < 1 and not math.copysign(1, x) < 0)
    # half uniform; a quarter random positive patterns, half of them below 1
    assert 0.57 < unit / len(xs) < 0.68
    assert any(x < 0 for x in xs) and any(abs(x) > 1e300 for x in xs)


def test_csv_rows_have_eight_columns():
    text = w.csv_columns_text(500, 8, 61)
    rows = text.split(b"\n")
    assert len(rows) == 500 and all(r.count(b",") == 7 for r in rows)


def test_packed_buffers_layout():
    texts = [b"1\n2", b"", b"3.5", b"x" * 40]
    arr, starts = w.pack_buffers(texts)
    for b, (s, t) in enumerate(zip(starts, texts)):
        assert s % 16 == b % 16
        assert bytes(arr[s:s + len(t)]) == t
    for (s0, t0), s1 in zip(zip(starts, texts), starts[1:]):
        assert s0 + len(t0) + 16 <= s1  # digits between neighbours
        assert set(bytes(arr[s0 + len(t0):s1])) == {ord("7")}


def test_midpoint_decimal_is_the_exact_midpoint():
    """The constructed midpoints the pins and parity tests use are exact:
    digits * 10^exp10 == (x + next(x)) / 2 in rational arithmetic, for
    normal and subnormal patterns, zero, and DBL_MAX (next = 2^1024)."""
    import struct
    from fractions import Fraction
    rng = np.random.Generator(np.random.PCG64(71))
    pats = [int(b) for b in rng.integers(0, 0x7FEFFFFFFFFFFFFF, size=400, dtype=np.int64)]
    pats += [0, 1, 0x000FFFFFFFFFFFFF, 0x0010000000000000, 0x7FEFFFFFFFFFFFFF]
    for b in pats:
        digits, e10 = w.midpoint_decimal(b)
        x = Fraction(struct.unpack("<d", struct.pack("<Q", b))[0])
        nxt = Fraction(2) ** 1024 if b == 0x7FEFFFFFFFFFFFFF else \
            Fraction(struct.unpack("<d", struct.pack("<Q", b + 1))[0])
        assert Fraction(int(digits)) * Fraction(10) ** e10 == (x + nxt) / 2, hex(b)
        assert not digits.endswith("0") or digits == "0"
