"""Pins of the oracle's field grammars and of the columnar layout rule.

* JSON: the JSON number grammar -- an optional '-', an integer part without
  leading zeros, an optional fraction with at least one digit, an optional
  exponent with at least one digit -- accepts exactly the forms it writes
  and rejects the others; an accepted number has the value the decimal
  grammar gives it.
* Hexadecimal floats (Appendix C): CPython's float.fromhex is correctly
  rounded and pins binary64 on random hexadecimal strings of every length
  and exponent, subnormal and overflowing ones included; for binary32 the
  nearest float by exact neighbour comparison; the paper's printed pairs
  (9000000000000000 = 0x1.ff973cafa8p+52, 5.972e24 = 0x1.3c27b13272fb6p+82).
* Columnar layout: hand-checked small CSV blocks, regular and ragged.
"""
import random
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
from test_oracle_f32_pins import INF32, nearest_f32

OK, INVALID, OVERFLOW, UNDERFLOW, BAD_SHAPE = 0, 1, 2, 3, 4
QNAN64 = 0x7FF8000000000000
HEX, JSON = oracle.GRAMMAR_HEX, oracle.GRAMMAR_JSON


def bits64(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


JSON_VALID = ["0", "-0", "1", "-1", "10", "907", "0.5", "-0.5", "0.0", "1.25", "1e5", "1E5",
              "1e+5", "1e-5", "0e0", "-0E-0", "123.456e-7", "1.7976931348623157e308",
              "4.9e-324", " 2.5", "2.5 ", "\t-3\r", "1" * 30, "0." + "0" * 40 + "1",
              "12345678901234567890123e-3"]
JSON_INVALID = ["+1", "01", "-01", "00", "0001.5", ".5", "-.5", "5.", "5.e3", "-", "", " ",
                "1e", "1e+", "1E-", "e5", "1.5.2", "--1", "1-", "0x10", "Infinity", "NaN",
                "1_000", "1,5", "1 2", "+0", "1.e5", "1ee5", "١"]


def test_json_grammar_accepts_exactly_the_json_forms():
    for s in JSON_VALID:
        got = oracle.parse_field_ex(s, grammar=JSON)
        assert got == oracle.parse_field(s), s       # the same number as the decimal grammar
        assert got[1] != INVALID, s
    for s in JSON_INVALID:
        assert oracle.parse_field_ex(s, grammar=JSON) == (QNAN64, INVALID), s


def test_json_grammar_on_random_forms():
    """Random strings from the decimal grammar: accepted under JSON exactly
    when they match the JSON number grammar (checked here by a regular
    expression written from that grammar), with the same value."""
    import re
    json_re = re.compile(r"^[ \t\r]*-?(0|[1-9][0-9]*)(\.[0-9]+)?([eE][+-]?[0-9]+)?[ \t\r]*$")
    rnd = random.Random(7)
    parts = ["", "+", "-"]
    for _ in range(40000):
        s = rnd.choice(parts) + "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(0, 4)))
        if rnd.random() < 0.6:
            s += "." + "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(0, 3)))
        if rnd.random() < 0.4:
            s += rnd.choice("eE") + rnd.choice(["", "+", "-"]) + \
                "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(0, 3)))
        got = oracle.parse_field_ex(s, grammar=JSON)
        if json_re.match(s):
            assert got == oracle.parse_field(s) and got[1] != INVALID, s
        else:
            assert got == (QNAN64, INVALID), s


def random_hex(rnd):
    digits = "".join(rnd.choice("0123456789abcdefABCDEF") for _ in range(rnd.randrange(1, 40)))
    cut = rnd.randrange(0, len(digits) + 1)
    body = digits[:cut] + ("." + digits[cut:] if rnd.random() < 0.7 else digits[cut:])
    if body == ".":
        body = "1"
    e = rnd.choice([rnd.randrange(-1100, 1100), rnd.randrange(-60, 60)])
    exp = ("p%+d" % e) if rnd.random() < 0.85 else ""
    sign = rnd.choice(["", "-", "+"])
    return sign + rnd.choice(["0x", "0X"]) + body + exp


def test_hex_matches_float_fromhex():
    rnd = random.Random(8)
    for _ in range(30000):
        s = random_hex(rnd)
        try:
            x = float.fromhex(s)
            want = (bits64(x), OK)
            mant = s.lstrip("+-")[2:].split("p")[0].split("P")[0]
            if x == 0 and any(c not in "0." for c in mant):
                want = (bits64(x), UNDERFLOW)   # nonzero digits rounded to zero
        except OverflowError:
            want = ((0x8000000000000000 if s.startswith("-") else 0) | 0x7FF0000000000000,
                    OVERFLOW)
        assert oracle.parse_field_ex(s, grammar=HEX) == want, s


def test_hex_binary32_by_neighbour_comparison():
    rnd = random.Random(9)
    for _ in range(5000):
        s = random_hex(rnd).lstrip("+-")
        body, _, e = s[2:].partition("p") if "p" in s else s[2:].partition("P")
        ip, _, fp_ = body.partition(".")
        v = Fraction(int((ip + fp_) or "0", 16)) * Fraction(2) ** (int(e or 0) - 4 * len(fp_))
        want = nearest_f32(v)
        got, st = oracle.parse_field_ex(s, f32=True, grammar=HEX)
        assert got == want, s
        assert st == (OVERFLOW if want == INF32 else (UNDERFLOW if want == 0 and v else OK)), s


def test_hex_examples_of_the_paper():
    # Appendix C prints these decimal / hexadecimal pairs
    for dec, hexs in (("9000000000000000", "0x1.ff973cafa8p+52"),
                      ("5.972e24", "0x1.3c27b13272fb6p+82")):
        assert oracle.parse_field_ex(hexs, grammar=HEX) == oracle.parse_field(dec)


def test_hex_grammar_edges():
    for s in ("0x", "0x.", "0xp3", "0x1p", "0x1p+", "1p3", "0x1.8q3", "0x1 .5", "0xg"):
        assert oracle.parse_field_ex(s, grammar=HEX)[1] == INVALID, s
    assert oracle.parse_field_ex("0x1.8", grammar=HEX) == (bits64(1.5), OK)   # no exponent
    assert oracle.parse_field_ex(" -0x0p0 ", grammar=HEX) == (0x8000000000000000, OK)
    assert oracle.parse_field_ex("0x1p-1075", grammar=HEX) == (0, UNDERFLOW)  # tie with zero
    assert oracle.parse_field_ex("0x1.8p-1074", grammar=HEX) == (2, OK)      # tie 1 | 2: even
    assert oracle.parse_field_ex("0x1.fffffffffffff8p1023", grammar=HEX)[1] == OVERFLOW
    assert oracle.parse_field_ex("0x1p3", grammar=oracle.GRAMMAR_DEFAULT)[1] == INVALID
    assert oracle.parse_field_ex("0x1p3", grammar=JSON)[1] == INVALID


def test_columnar_layout_by_hand():
    text = b"1,2,3\n4,5,6\n7,8,9"
    bits, st = oracle.parse_buffer(text, b",")
    out, ost = oracle.columnar(text, bits, st, 3, 4)
    vals = out.view(np.float64)
    assert list(vals[0:3]) == [1, 4, 7] and list(vals[4:7]) == [2, 5, 8] and \
        list(vals[8:11]) == [3, 6, 9]
    assert (ost[[0, 1, 2, 4, 5, 6, 8, 9, 10]] == OK).all() and (ost[[3, 7, 11]] == 0xEE).all()
    # a short row: its last field ends at '\n' in column 1; the rows after it
    # are off by one, so the fields that meet a wrong terminator are flagged
    text = b"1,2,3\n4,5\n7,8,9\n"
    bits, st = oracle.parse_buffer(text, b",")
    out, ost = oracle.columnar(text, bits, st, 3, 3)
    # fields: 1 2 3 | 4 5 | 7 8 9 -> indices 0..7; 5 (index 4, column 1) ends at '\n',
    # 7 (index 5, column 2) ends at ',', 9 (index 7, column 1) ends at '\n'
    flagged = sorted(int(i) for i in np.nonzero(ost == BAD_SHAPE)[0])
    dest = lambda i: (i % 3) * 3 + i // 3
    assert flagged == sorted([dest(4), dest(5), dest(7)])
    assert out.view(np.float64)[dest(6)] == 8.0


def test_paper_grammar_examples():
    """The grammar examples printed in Section 4 (tests/golden/grammar_examples.txt)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "grammar_examples.txt")
    n = 0
    with open(path) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            text, grammar, expected, _ = ln.rstrip("\n").split("\t")
            g = JSON if grammar == "json" else oracle.GRAMMAR_DEFAULT
            got = oracle.parse_field_ex(text, grammar=g)
            if expected == "INVALID":
                assert got == (QNAN64, INVALID), text
            else:
                assert got == (bits64(float(expected)), OK), text
                # and JSON rejects none of the plain spellings it allows
            n += 1
    assert n == 10


def test_hex_float_text_round_trips():
    """Appendix C's hexadecimal floats are dyadic, so parsing float.hex(x)
    gives x exactly (Python's own conversion, independent of the oracle);
    to binary32 it gives the one rounding of that exact value (numpy's),
    with overflow to infinity and underflow to zero flagged.  Uniform
    values, random finite bit patterns of both signs, subnormals, zeros."""
    import numpy as np
    from paper_2101_11408_gb300 import workloads
    lines = workloads.hex_float_lines(20000, 91) + [
        (5e-324).hex(), (-5e-324).hex(), (2.2250738585072014e-308).hex(), (0.0).hex(),
        (-0.0).hex(), (1.7976931348623157e308).hex()]
    text = "\n".join(lines).encode()
    xs = np.array([float.fromhex(s) for s in lines])
    bits, st = oracle.parse_buffer(text, grammar=oracle.GRAMMAR_HEX)
    assert np.array_equal(bits, xs.view(np.uint64))
    assert (st == 0).all()
    b32, s32 = oracle.parse_buffer(text, f32=True, grammar=oracle.GRAMMAR_HEX)
    with np.errstate(over="ignore", under="ignore"):
        want = xs.astype(np.float32)
    assert np.array_equal(b32, want.view(np.uint32))
    want_st = np.where(np.isinf(want), 2, np.where((want == 0) & (xs != 0), 3, 0))
    assert np.array_equal(s32, want_st.astype(np.uint8))
