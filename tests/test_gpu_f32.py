"""GPU parity of fp_parse_f32 (binary32 results) against the oracle's
binary32 conversion, bit for bit: values, statuses and field counts.  The
inputs are the binary64 suite's shapes plus binary32's own hard cases
(float32 round trips, midpoints between adjacent floats, the binary32
range boundaries)."""
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import workloads
from test_gpu_parity import join, to_device
from test_oracle_f32_pins import bump_last_digit, exact_decimal, f32_value, random_finite_f32

pytestmark = pytest.mark.gpu


def gpu_parse32(text: bytes, delim=b"\n", offset=0):
    t = to_device(text, offset)
    vals, st = fp.parse_f32(t, delim)
    torch.cuda.synchronize()
    assert fp.get_error() == 0
    return vals.cpu().numpy().view(np.uint32), st.cpu().numpy()


def assert_parity32(text: bytes, delim=b"\n", offset=0, lines=None):
    bits, st = gpu_parse32(text, delim, offset)
    rb, rs = oracle.parse_buffer(text, delim, f32=True)
    assert bits.size == rb.size, "field count %d vs oracle %d" % (bits.size, rb.size)
    bad = np.nonzero((bits != rb) | (st != rs))[0]
    if bad.size:
        i = int(bad[0])
        what = lines[i][:80] if lines is not None and i < len(lines) else "?"
        pytest.fail("%d mismatches; first at field %d %r: gpu %#x/%d oracle %#x/%d" % (
            bad.size, i, what, int(bits[i]), int(st[i]), int(rb[i]), int(rs[i])))
    return bits, st


def test_float32_round_trips():
    rnd = random.Random(61)
    lines = []
    for b in random_finite_f32(rnd, 60000):
        x = np.array([b], dtype=np.uint32).view(np.float32)[0]
        lines += ["%.9g" % float(x), np.format_float_scientific(x, unique=True),
                  "-" + np.format_float_positional(x, unique=True)]
    bits, _ = assert_parity32(join(lines), lines=lines)
    assert (bits[0::3] == np.array(random_finite_f32(random.Random(61), 60000),
                                   dtype=np.uint32)).all()


def test_float32_midpoints_and_neighbours():
    rnd = random.Random(62)
    lines = []
    for b in random_finite_f32(rnd, 8000, subnormal_share=0.3) + [1, 2, 0x7FFFFF, 0x800000,
                                                                 0x7F7FFFFE]:
        s = exact_decimal((f32_value(b) + f32_value(b + 1)) / 2)
        lines += [s, bump_last_digit(s, 1), bump_last_digit(s, -1)]
    mid = (f32_value(0x7F7FFFFF) + Fraction(2) ** 128) / 2
    lines += [exact_decimal(mid), bump_last_digit(exact_decimal(mid), -1)]
    assert_parity32(join(lines), lines=lines)


def test_small_significands_all_exponents():
    lines = ["%de%d" % (m, e) for m in range(1, 1000) for e in range(-70, 50)]
    assert_parity32(join(lines), lines=lines)


def test_binary32_boundaries_and_grammar():
    from test_oracle_pins import GRAMMAR
    lines = [g for g, _ in GRAMMAR if "\n" not in g] + [
        "3.4028235e38", "3.4028236e38", "-3.40282356779733661637539395458142568448e38",
        "1e-45", "7e-46", "7.1e-46", "1.17549435e-38", "1.1754942e-38", "16777217",
        "16777219", "1e10", "1e11", "0.1", "-0", "1e39", "1e-46", "0." + "0" * 50 + "1"]
    assert_parity32(join(lines), lines=lines)


def test_random_strings():
    from test_oracle_pins import _random_strings
    lines = _random_strings(random.Random(63), 100000)
    assert_parity32(join(lines), lines=lines)


def test_workloads():
    assert_parity32(workloads.uniform_text(10000))
    assert_parity32(workloads.bulk_mixed_text(1_000_000, 64))
    assert_parity32(workloads.hard_case_text(100_000, 65))


def test_bulk_mixed_10m():
    text = workloads.bulk_mixed_text()
    bits, _ = assert_parity32(text)
    assert bits.size == 10_000_000


@pytest.mark.parametrize("chunk", [4096, 8192, 12288, 16384])
def test_chunk_sizes_and_unaligned_starts(chunk):
    before = fp.get_config()
    try:
        fp.set_config(chunk_bytes=chunk)
        text = workloads.bulk_mixed_text(200000, 66)
        for offset in (0, 5, 15):
            assert_parity32(text, offset=offset)
        assert_parity32(workloads.hard_case_text(20000, 67))
    finally:
        fp.set_config(**before)


def test_queue_overflow_path_reads_locations_from_the_side_array():
    before = fp.get_config()
    try:
        fp.set_config(fallback_queue=1024)
        fp.stats(reset=True)
        lines = workloads.hard_case_lines(30000, 68)
        assert_parity32(join(lines), lines=lines)
        assert fp.stats()["queue_overflow"] > 0
    finally:
        fp.set_config(**before)


def test_comma_delimiter_and_empty_buffers():
    rows = [",".join(workloads.uniform_lines(8, s)) for s in range(2000)]
    assert_parity32("\n".join(rows).encode(), delim=b",")
    for text in [b"", b"\n", b"\n\n", b"1", b"1\n\n2\n", b" \n \n"]:
        assert_parity32(text)


def test_f32_and_f64_calls_interleave_on_one_stream():
    a = workloads.hard_case_text(5000, 69)
    b = workloads.bulk_mixed_text(50000, 70)
    for _ in range(2):
        assert_parity32(a)
        v, s = fp.parse_f64(to_device(a))
        rb, rs = oracle.parse_buffer(a)
        assert np.array_equal(v.cpu().numpy().view(np.uint64), rb)
        assert_parity32(b)


def test_integer_file_to_binary32():
    """Integer files to binary32: 32- to 64-bit integers rounded to 24 bits,
    to nearest with ties to even (and the ties just above 2^24)."""
    lines = workloads.integer_lines(1_000_000, 141) + [str((1 << 24) + k) for k in range(64)]
    assert_parity32("\n".join(lines).encode(), lines=lines)
