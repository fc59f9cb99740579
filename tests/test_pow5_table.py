"""The 128-bit power-of-five table used by the GPU path, against the paper.

The table is data for the CUDA kernels (the oracle uses no table).  These
tests pin the generator to the rows the paper prints (Tables pospower,
tabnearone, awayfromone, insane) and to the closed-form claims around it.
"""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2101_11408_gb300", "csrc")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_pow5_table",
                                                  os.path.join(CSRC, "gen_pow5_table.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


gen = _gen()
M64 = (1 << 64) - 1


def test_generated_include_is_current():
    with open(os.path.join(CSRC, "pow5_table.inc")) as f:
        assert f.read() == gen.render()


def test_table_size():
    """651 entries of 16 bytes (Section 12 quotes about 10 KiB)."""
    t = gen.table()
    assert len(t) == 651 and 16 * len(t) == 10416


def _rows(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.mark.parametrize("row", _rows("pow5_table_rows.txt"), ids=lambda r: "%s%s" % (r[0], r[1]))
def test_printed_rows(row):
    kind, q, first, second = row[0], int(row[1]), int(row[2], 16), int(row[3], 16)
    v = gen.table_entry(q)
    assert v >> 64 == first
    assert v & M64 == second


def test_every_entry_is_normalised():
    for q in range(-342, 309):
        v = gen.table_entry(q)
        assert (1 << 127) <= v < (1 << 128), q


def test_positive_powers_exact_up_to_55():
    """Section 8: 5^q < 2^128 for q <= 55, so the stored 128 bits are exact."""
    for q in range(0, 56):
        v = gen.table_entry(q)
        p = 5 ** q
        assert v == p << (128 - p.bit_length())
    assert 5 ** 55 < (1 << 128) <= 5 ** 56


def test_near_reciprocals_are_ceilings():
    """Section 9.1: c = ceil(2^b / 5^-q), b = 127 + ceil(log2 5^-q)."""
    for q in range(-27, 0):
        d = 5 ** (-q)
        c = gen.table_entry(q)
        b = 127 + (d - 1).bit_length()
        assert (c - 1) * d < (1 << b) <= c * d


def _newton_inverse(x):
    """Multiplicative inverse of an odd 64-bit word by Newton's iteration
    (Appendix "Multiplicative Inverses": y <- y (2 - y x), five steps)."""
    y = x
    for _ in range(5):
        y = (y * (2 - y * x)) & M64
    return y


@pytest.mark.parametrize("row", _rows("inverse_table_rows.txt"), ids=lambda r: r[0])
def test_insane_table(row):
    """Table insane: no false tie after one multiplication."""
    q, hi, inv, prod, tz = int(row[0]), int(row[1], 16), int(row[2], 16), int(row[3], 16), int(row[4])
    assert gen.table_entry(q) >> 64 == hi
    y = _newton_inverse(hi)
    assert y == inv and (hi * y) & M64 == 1
    ph = (hi * y) >> 64
    assert ph == prod
    assert (ph & -ph).bit_length() - 1 == tz <= 5


def test_near_high_words_have_few_trailing_zeros():
    """Section 9.1: the high words for q in [-17,-1] have at most 2 trailing
    zeros, and the odd ones are exactly the rows of Table insane."""
    odd = []
    for q in range(-17, 0):
        hi = gen.table_entry(q) >> 64
        assert (hi & -hi).bit_length() - 1 <= 2
        if hi & 1:
            odd.append(q)
    assert sorted(odd) == sorted(int(r[0]) for r in _rows("inverse_table_rows.txt"))


def test_exponent_formula():
    """Section 10: (217706 q) >> 16 == q + floor(log2 5^q) == floor(log2 10^q)
    for every q in (-400, 350)."""
    for q in range(-399, 350):
        if q >= 0:
            exact = (10 ** q).bit_length() - 1
        else:
            exact = -((10 ** (-q) - 1).bit_length())
        assert (217706 * q) >> 16 == exact, q
