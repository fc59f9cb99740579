"""The fallback kernel's tables of powers of five and two in base 10^9
(gen_dec_tables.py): the committed include matches the generator, every
entry is the exact power, and the ranges cover every midpoint a binary64
or binary32 comparison needs (5^j for j <= 1075, 2^k for k <= 970)."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2101_11408_gb300", "csrc")


@pytest.fixture(scope="module")
def gen():
    spec = importlib.util.spec_from_file_location("gen_dec_tables",
                                                  os.path.join(CSRC, "gen_dec_tables.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_include_is_current(gen):
    with open(os.path.join(CSRC, "dec_tables.inc")) as f:
        assert f.read() == gen.render()


def test_entries_are_exact_powers(gen):
    for base, step, count in ((5, gen.DEC5_STEP, gen.DEC5_COUNT), (2, gen.DEC2_STEP, gen.DEC2_COUNT)):
        offs, data = gen.table(base, step, count)
        assert len(offs) == count + 1 and offs[-1] == len(data)
        for a in range(count):
            limbs = data[offs[a]:offs[a + 1]]
            assert all(0 <= v < 10 ** 9 for v in limbs) and limbs[-1] != 0
            assert sum(v * 10 ** (9 * i) for i, v in enumerate(limbs)) == base ** (step * a)


def test_ranges_cover_every_midpoint(gen):
    # binary64: e = 1 - 1075 .. 2046 - 1075; the kernel uses 5^(1-e) for
    # e <= 0 and 2^(e-1) for e >= 1, as table entry * a power below the step
    assert (1075 // gen.DEC5_STEP) < gen.DEC5_COUNT
    assert (970 // gen.DEC2_STEP) < gen.DEC2_COUNT
    assert 5 ** (gen.DEC5_STEP - 1) < 10 ** 9 and 2 ** (gen.DEC2_STEP - 1) < 10 ** 9
