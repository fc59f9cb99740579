"""The oracle against glibc's strtod, a second correctly rounded conversion
written independently of it (besides CPython's float(), used by
test_oracle_pins): random decimal strings of 1 to 120 digits, the hard-case
mix (up to 800 digits, exact midpoints and their neighbours, the ends of
the range), all through ctypes in the "C" locale, round to nearest."""
import ctypes
import ctypes.util
import random
import struct

import numpy as np
import pytest

import oracle
from paper_2101_11408_gb300 import workloads
from test_oracle_pins import _random_strings


@pytest.fixture(scope="module")
def strtod():
    name = ctypes.util.find_library("c")
    if not name:
        pytest.skip("no C library")
    libc = ctypes.CDLL(name)
    if not hasattr(libc, "gnu_get_libc_version"):
        pytest.skip("not glibc (whose strtod is correctly rounded)")
    f = libc.strtod
    f.restype = ctypes.c_double
    f.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_char_p)]
    return f


def _bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _compare(strtod, lines):
    text = "\n".join(lines).encode()
    rb, rs = oracle.parse_buffer(text)
    assert rb.size == len(lines)
    for i, s in enumerate(lines):
        want = _bits(strtod(s.encode(), None))
        assert int(rb[i]) == want, (s[:80], hex(int(rb[i])), hex(want))
        assert rs[i] in (0, 2, 3)


def test_random_decimal_strings(strtod):
    _compare(strtod, _random_strings(random.Random(2101), 60000))


def test_hard_cases(strtod):
    _compare(strtod, workloads.hard_case_lines(6000, workloads.SEED_BASE + 61))


def test_midpoints_and_neighbours(strtod):
    rng = np.random.Generator(np.random.PCG64(62))
    lines = []
    for b in rng.integers(0, 0x7FEFFFFFFFFFFFFF, size=3000, dtype=np.int64).tolist():
        d, e = workloads.midpoint_decimal(int(b))
        for delta in (0, 1, -1):
            lines.append("%se%d" % (int(d) + delta, e))
    _compare(strtod, lines)
