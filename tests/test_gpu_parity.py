"""GPU parity: the CUDA path against the CPU oracle, bit for bit.

Every test feeds the same seeded text to the library (through the C ABI)
and to the oracle, and requires identical binary64 bit patterns, identical
status bytes and identical field counts (the result is exact integer and bit
work, so the tolerance is zero).
"""
import os
import random

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def to_device(text: bytes, offset: int = 0, guard: int = 48, junk: int = ord("7")):
    """Device copy of text starting `offset` bytes into an allocation whose
    other bytes are `junk` (digits, so that any use of them would show)."""
    buf = torch.full((guard + offset + len(text) + guard,), junk, dtype=torch.uint8)
    if text:
        buf[guard + offset: guard + offset + len(text)] = torch.frombuffer(bytearray(text),
                                                                           dtype=torch.uint8)
    dev = buf.cuda()
    return dev[guard + offset: guard + offset + len(text)]


def gpu_parse(text: bytes, delim=b"\n", offset=0):
    t = to_device(text, offset)
    vals, st = fp.parse_f64(t, delim)
    torch.cuda.synchronize()
    assert fp.get_error() == 0
    return vals.cpu().numpy().view(np.uint64), st.cpu().numpy()


def assert_parity(text: bytes, delim=b"\n", offset=0, lines=None):
    bits, st = gpu_parse(text, delim, offset)
    rb, rs = oracle.parse_buffer(text, delim)
    assert bits.size == rb.size, "field count %d vs oracle %d" % (bits.size, rb.size)
    bad = np.nonzero((bits != rb) | (st != rs))[0]
    if bad.size:
        i = int(bad[0])
        what = lines[i][:80] if lines is not None and i < len(lines) else "?"
        pytest.fail("%d mismatches; first at field %d %r: gpu %#x/%d oracle %#x/%d" % (
            bad.size, i, what, int(bits[i]), int(st[i]), int(rb[i]), int(rs[i])))
    return bits, st


def join(lines, sep="\n"):
    return sep.join(lines).encode("utf-8")


# --------------------------------------------------------------------------
# small, exhaustive and adversarial inputs
# --------------------------------------------------------------------------

def test_paper_examples():
    lines = []
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                lines.append(ln.split("\t")[0])
    assert_parity(join(lines), lines=lines)


def test_grammar_and_edge_fields():
    from test_oracle_pins import GRAMMAR
    lines = [g for g, _ in GRAMMAR if "\n" not in g] + [
        "-0", "+0", "0e999999999999", "1e-400", "-1e400", "9007199254740993",
        "2.2250738585072014e-308", "4.9406564584124654e-324", "1.7976931348623157e308",
        "1.7976931348623159e308", "0." + "0" * 60 + "1", "1" + "0" * 40, " ", "\t-.5\r"]
    assert_parity(join(lines), lines=lines)


def test_random_strings():
    from test_oracle_pins import _random_strings
    lines = _random_strings(random.Random(77), 150000)
    assert_parity(join(lines), lines=lines)


def test_small_significands_all_exponents():
    lines = ["%de%d" % (m, e) for m in range(1, 1000) for e in range(-345, 311)]
    assert_parity(join(lines), lines=lines)


def test_constructed_midpoints():
    rng = np.random.Generator(np.random.PCG64(21))
    bits = [int(b) for b in rng.integers(0, 0x7FEFFFFFFFFFFFFF, size=20000, dtype=np.int64)]
    bits += [0, 1, 0x000FFFFFFFFFFFFF, 0x0010000000000000, 0x7FEFFFFFFFFFFFFE, 0x7FEFFFFFFFFFFFFF]
    lines = []
    for b in bits:
        d, e = workloads.midpoint_decimal(b)
        for delta in (0, 1, -1):
            lines.append("%se%d" % (int(d) + delta, e))
    assert_parity(join(lines), lines=lines)


def test_empty_and_separator_only_buffers():
    for text in [b"", b"\n", b"\n\n\n", b"1", b"1\n", b"\n1", b"1\n\n2\n", b" \n \n"]:
        assert_parity(text)


def test_comma_delimiter():
    rows = [",".join(workloads.uniform_lines(8, s)) for s in range(3000)]
    text = "\n".join(rows).encode()
    assert_parity(text, delim=b",")
    # with '\n' as the only separator every row is one (invalid) field
    assert_parity(text, delim=b"\n")


def test_unaligned_pointers_and_guard_bytes():
    lines = workloads.bulk_mixed_lines(3000, 8)
    text = join(lines)
    for offset in range(16):
        for cut in (1, 2, 15, 16, 17, 31, 100, 1000, len(text)):
            assert_parity(text[:cut], offset=offset)


@pytest.mark.parametrize("chunk", [4096, 8192, 12288, 16384])
def test_fields_straddling_chunks(chunk):
    before = fp.get_config()
    try:
        fp.set_config(chunk_bytes=chunk)
        rnd = random.Random(chunk)
        lines = []
        for _ in range(40000):
            k = rnd.randrange(6)
            if k == 0:
                lines.append("%.17g" % rnd.random())
            elif k == 1:
                lines.append(str(rnd.randrange(10 ** rnd.randrange(1, 20))))
            elif k == 2:  # around the short-field limit
                n = rnd.randrange(55, 75)
                lines.append("1." + "".join(rnd.choice("0123456789") for _ in range(n - 2)))
            elif k == 3:
                lines.append("")
            elif k == 4:
                n = rnd.randrange(20, 300)
                lines.append("".join(rnd.choice("0123456789") for _ in range(n)) + "e-%d" % n)
            else:
                lines.append(" %se%d " % (rnd.randrange(1, 99999), rnd.randrange(-330, 310)))
        text = join(lines)
        for offset in (0, 3):
            assert_parity(text, offset=offset, lines=lines)
    finally:
        fp.set_config(**before)


def test_long_fields():
    rnd = random.Random(5)
    lines = []
    for n in list(range(60, 70)) + [100, 777, 800, 801, 1000, 5000, 100000]:
        d = rnd.choice("123456789") + "".join(rnd.choice("0123456789") for _ in range(n - 1))
        lines.append(d[:3] + "." + d[3:] + "e-%d" % rnd.randrange(0, 300))
        lines.append("0." + "0" * n + "1e%d" % (n + 1))  # exactly 1
        lines.append("1" + "0" * n)  # 1e(n): inf beyond 308
    assert_parity(join(lines), lines=lines)


def _long_defects(rnd, count):
    """Fields longer than the parse kernel's 64-byte limit (the fallback
    kernel's), most with one defect -- a stray byte, a second point, a
    blank, a sign, an empty or broken exponent -- at an offset on or next to
    the fallback pass's 32- and 64-byte round boundaries, and valid
    controls, leading zeros and points included."""
    spots = [0, 1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 127, 128, 129, 191, 192, 193]
    out = []
    for _ in range(count):
        n = rnd.randrange(66, 260)
        d = "".join(rnd.choice("0123456789") for _ in range(n))
        if rnd.random() < 0.3:
            d = "0" * rnd.randrange(1, 40) + d
        if rnd.random() < 0.6:
            p = rnd.randrange(0, len(d) + 1)
            d = d[:p] + "." + d[p:]
        k = rnd.randrange(8)
        at = min(rnd.choice(spots + [rnd.randrange(0, len(d))]), len(d) - 1)
        if k == 0:
            f = d[:at] + rnd.choice("x/:-+ ,") + d[at + 1:]
        elif k == 1:
            f = d[:at] + "." + d[at:]
        elif k == 2:
            f = d + rnd.choice(["e", "E", "e+", "e-", "e1x", "e--1", "ee1", "e 1"])
        elif k == 3:
            f = d[:at] + "e" + d[at:]  # the marker mid-significand: the rest is the exponent
        elif k == 4:
            f = d + "e" + str(rnd.randrange(-400, 400))
        elif k == 5:
            f = rnd.choice(["", "-", "+", " ", "\t"]) + d + rnd.choice(["", " ", "\r"])
        elif k == 6:
            f = d[:at] + "\t" + d[at:]
        else:
            f = d
        out.append(f)
    return out


def test_long_malformed_fields():
    """The fallback kernel's grammar checks agree with the oracle's on long
    fields, valid or with one defect near its pass's round boundaries."""
    lines = _long_defects(random.Random(123), 12000)
    assert_parity(join(lines), lines=lines)


def test_long_fields_json_grammar():
    """The JSON number grammar on long fields (the fallback kernel's copy of
    its rules): leading zeros, a point with no digit on one side, '+'."""
    rnd = random.Random(124)
    lines = _long_defects(rnd, 4000)
    for _ in range(2000):
        d = "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(66, 200)))
        lines += ["0" + d, "-0" + d, "0." + d, "." + d, d + ".", d + ".e5", "+" + d,
                  d[:5] + "." + d[5:] + "E+12", "-" + d + "e-7"]
    text = join(lines)
    t = to_device(text)
    vals, st = fp.parse_ex(t, grammar="json")
    rb, rs = oracle.parse_buffer(text, grammar=oracle.GRAMMAR_JSON)
    got = vals.cpu().numpy().view(np.uint64)
    assert got.size == rb.size
    bad = np.nonzero((got != rb) | (st.cpu().numpy() != rs))[0]
    assert bad.size == 0, "first mismatch at %r" % lines[int(bad[0])][:90]


def test_huge_single_field():
    """A 16 MB field: 1 + 10^-16M rounds to 1.0; its integer twin overflows."""
    n = 16 << 20
    text = b"1." + b"0" * n + b"1"
    bits, st = gpu_parse(text)
    assert bits.tolist() == [0x3FF0000000000000] and st.tolist() == [0]
    text = b"1" + b"3" * n + b"\n-0." + b"0" * n + b"7"
    bits, st = gpu_parse(text)
    assert bits.tolist() == [0x7FF0000000000000, 1 << 63]
    assert st.tolist() == [fp.STATUS_OVERFLOW, fp.STATUS_UNDERFLOW]


# --------------------------------------------------------------------------
# the paper-shaped workloads
# --------------------------------------------------------------------------

def test_uniform_10k():
    text = workloads.uniform_text(10000)
    assert_parity(text)


def test_bulk_mixed_10m():
    text = workloads.bulk_mixed_text(10_000_000)
    bits, st = assert_parity(text)
    assert bits.size == 10_000_000


def test_hard_cases_1m():
    text = workloads.hard_case_text(1_000_000)
    bits, st = assert_parity(text)
    assert bits.size == 1_000_000


def test_queue_overflow_path():
    """A fallback queue far smaller than the number of fallback fields: the
    rest are found by scanning their chunks, with identical results."""
    before = fp.get_config()
    try:
        fp.set_config(fallback_queue=1024)
        fp.stats(reset=True)
        lines = workloads.hard_case_lines(30000, 99)
        assert_parity(join(lines), lines=lines)
        assert fp.stats()["queue_overflow"] > 0
    finally:
        fp.set_config(**before)


@pytest.mark.parametrize("chunk", [4096, 8192, 12288, 16384])
@pytest.mark.parametrize("per_sm", [1, 0])
def test_launch_configurations(chunk, per_sm):
    before = fp.get_config()
    try:
        fp.set_config(chunk_bytes=chunk, ctas_per_sm=per_sm)
        assert_parity(workloads.bulk_mixed_text(300000, 31))
    finally:
        fp.set_config(**before)


def test_repeated_calls_reset_state():
    texts = [workloads.bulk_mixed_text(50000 + 1000 * i, 40 + i) for i in range(4)]
    texts += [b"", b"1\n2", workloads.hard_case_text(5000, 3)]
    for t in texts * 2:
        assert_parity(t)


def test_two_streams_concurrently():
    a = workloads.bulk_mixed_text(400000, 51)
    b = workloads.hard_case_text(20000, 52)
    ta, tb = to_device(a), to_device(b)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for t, s in ((ta, sa), (tb, sb)):
        out = torch.empty(t.numel(), dtype=torch.float64, device="cuda")
        st = torch.empty(t.numel(), dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        fp.parse_f64_into(t, out, st, cnt, stream=s)
        outs.append((out, st, cnt))
    torch.cuda.synchronize()
    for (out, st, cnt), text in zip(outs, (a, b)):
        n = int(cnt.item())
        rb, rs = oracle.parse_buffer(text)
        assert n == rb.size
        assert np.array_equal(out[:n].cpu().numpy().view(np.uint64), rb)
        assert np.array_equal(st[:n].cpu().numpy(), rs)


def test_stats_path_frequencies():
    """Table percentage: on uniform data about 0.66% of the numbers need the
    second product and none needs the fallback (loose band, not parity)."""
    text = workloads.uniform_text(1_000_000, 61)
    fp.stats(reset=True)
    gpu_parse(text)
    s = fp.stats(reset=True)
    assert s["fields"] == 1_000_000
    rate = s["two_multiplies"] / s["fields"]
    assert 0.002 < rate < 0.015, rate
    assert s["fallback"] == 0


def test_long_check_settles_most():
    """Section 11: truncating to 19 digits and checking w and w+1 settles
    about 99.7-99.8% of long random significands."""
    rnd = random.Random(8)
    lines = []
    for _ in range(100000):
        d = rnd.choice("123456789") + "".join(rnd.choice("0123456789") for _ in range(24))
        lines.append("%s.%se%d" % (d[:1], d[1:], rnd.randrange(-300, 300)))
    fp.stats(reset=True)
    assert_parity(join(lines), lines=lines)
    s = fp.stats(reset=True)
    assert s["long_fields"] == 100000
    assert s["long_settled"] / s["long_fields"] > 0.99


# --------------------------------------------------------------------------
# batched entry point
# --------------------------------------------------------------------------

def test_batch_matches_single_and_oracle():
    rnd = random.Random(3)
    texts = []
    for i in range(60):
        k = rnd.randrange(4)
        if k == 0:
            texts.append(b"")
        elif k == 1:
            texts.append(workloads.uniform_text(rnd.randrange(1, 3000), 100 + i))
        elif k == 2:
            texts.append(workloads.bulk_mixed_text(rnd.randrange(1, 20000), 200 + i))
        else:
            texts.append(workloads.hard_case_text(rnd.randrange(1, 500), 300 + i))
    dev = [to_device(t, offset=i % 16) for i, t in enumerate(texts)]
    res = fp.parse_f64_batch(dev)
    for t, (v, s) in zip(texts, res):
        rb, rs = oracle.parse_buffer(t)
        assert v.numel() == rb.size
        assert np.array_equal(v.cpu().numpy().view(np.uint64), rb)
        assert np.array_equal(s.cpu().numpy(), rs)


def test_batch_capacity_limits_writes():
    text = workloads.uniform_text(1000, 7)
    t = to_device(text)
    out = torch.full((600,), -1.0, dtype=torch.float64, device="cuda")
    st = torch.full((600,), 9, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    fp.parse_f64_batch_into([t, t], out, st, [0, 100, 300], cnt)
    torch.cuda.synchronize()
    assert cnt.cpu().tolist() == [1000, 1000]
    rb, _ = oracle.parse_buffer(text)
    got = out.cpu().numpy().view(np.uint64)
    assert np.array_equal(got[:100], rb[:100])
    assert np.array_equal(got[100:300], rb[:200])
    assert (out[300:].cpu() == -1.0).all() and (st[300:].cpu() == 9).all()


def test_host_entry_point():
    text = workloads.bulk_mixed_text(20000, 71)
    vals, st = fp.parse_f64_host(text)
    rb, rs = oracle.parse_buffer(text)
    assert np.array_equal(vals.view(np.uint64), rb) and np.array_equal(st, rs)


def test_host_entry_point_direct():
    """Below 8 MB with pinned result arrays the parse kernel writes the
    results and the count into host memory itself: equal to the oracle,
    hard cases included (the fallback kernel then reads the pending fields'
    locations from, and writes their values to, the pinned arrays), nothing
    written past the count, for pinned and pageable text."""
    texts = [workloads.bulk_mixed_text(100_000, 94), workloads.hard_case_text(5_000, 95), b"",
             b"1", b"\n\n", b"1e-400\n-0\nx\n" + b"9" * 900 + b"e-1000"]
    for text in texts:
        rb, rs = oracle.parse_buffer(text)
        n = len(text) + 64
        for pin_text in (True, False):
            h_text = (torch.frombuffer(bytearray(text), dtype=torch.uint8) if text
                      else torch.empty(0, dtype=torch.uint8))
            if pin_text:
                h_text = h_text.pin_memory()
            h_out = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
            h_st = torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory()
            k = fp.parse_f64_host_into(h_text, h_out, h_st)
            assert k == rb.size, (text[:30], pin_text)
            assert np.array_equal(h_out[:k].numpy().view(np.uint64), rb)
            assert np.array_equal(h_st[:k].numpy(), rs)
            assert (h_st[k:].numpy() == 0xEE).all() and (h_out[k:].numpy() == -1.0).all()
    assert fp.get_error() == 0


def test_autotune_picks_a_valid_config(tmp_path):
    import json
    before = fp.get_config()
    try:
        path = str(tmp_path / "tune.json")
        bulk = to_device(workloads.bulk_mixed_text(200000, 81))
        c = fp.autotune(bulk, cache_path=path)
        assert c["chunk_bytes"] in (4096, 8192, 12288, 16384)
        assert c["ctas_per_sm"] in (0, 1, 2, 3, 4)
        assert c["fallback_queue"] in (1 << 16, 1 << 18, 1 << 20, 1 << 22)
        fp.set_config(**before)
        c2 = fp.autotune(bulk, cache_path=path)  # loaded from the cache
        assert c2 == c
        # another class of workload (most fields pending) gets its own entry
        hard = to_device(workloads.hard_case_text(200000, 83))
        fp.set_config(**before)
        c3 = fp.autotune(hard, cache_path=path)
        assert c3["fallback_queue"] in (1 << 16, 1 << 18, 1 << 20, 1 << 22)
        with open(path) as f:
            entries = [json.loads(line) for line in f if line.strip()]
        classes = sorted(e["class"] for e in entries)
        assert len(entries) == 2 and classes[0] != classes[1], entries
        assert any("fallback=many" in k for k in classes) and any("fallback=rare" in k for k in classes)
        fp.set_config(**before)
        assert fp.autotune(bulk, cache_path=path) == c  # the first entry is still there
        assert_parity(workloads.bulk_mixed_text(50000, 82))
    finally:
        fp.set_config(**before)


@pytest.mark.parametrize("delim", [b"\n", b","])
def test_host_entry_point_pipelined(delim):
    """Texts of 32 MB and more in pinned memory take the pipelined path
    (segments cut at separators, parsed as they arrive, their results
    copied back at the running field total); they must equal the oracle,
    and pageable copies of the same arrays (the one-copy path)."""
    parts = [workloads.bulk_mixed_text(1_500_000, 91), workloads.hard_case_text(20_000, 92),
             b"7" * (3 << 20),  # a field of 3 MB: no separator near some cuts
             workloads.bulk_mixed_text(800_000, 93)]
    text = b"\n".join(parts)
    if delim == b",":
        text = text.replace(b"\n", b",", 200_000)
    n = len(text)
    rb, rs = oracle.parse_buffer(text, delim)
    for pinned in (True, False):
        h_text = torch.frombuffer(bytearray(text), dtype=torch.uint8)
        h_out = torch.full((n,), -1.0, dtype=torch.float64)
        h_st = torch.full((n,), 0xEE, dtype=torch.uint8)
        if pinned:
            h_text, h_out, h_st = h_text.pin_memory(), h_out.pin_memory(), h_st.pin_memory()
        k = fp.parse_f64_host_into(h_text, h_out, h_st, delim)
        assert k == rb.size
        assert np.array_equal(h_out[:k].numpy().view(np.uint64), rb)
        assert np.array_equal(h_st[:k].numpy(), rs)
        assert (h_st[k:k + 1000].numpy() == 0xEE).all()  # nothing written past the count
    assert fp.get_error() == 0


def test_host_entry_point_pipelined_tapered_segments():
    """A text of about 80 MB in pinned memory: full segments, then three
    shrinking ones, each segment's results copied back at the running field
    total; hard cases (fields for the fallback kernel) sit in the first and
    in the last, smallest segments."""
    parts = [workloads.hard_case_text(5_000, 135), workloads.bulk_mixed_text(4_000_000, 136),
             workloads.hard_case_text(5_000, 137)]
    text = b"\n".join(parts)
    assert len(text) > (72 << 20)
    n = len(text)
    rb, rs = oracle.parse_buffer(text)
    h_text = torch.frombuffer(bytearray(text), dtype=torch.uint8).pin_memory()
    h_out = torch.full((n,), -1.0, dtype=torch.float64).pin_memory()
    h_st = torch.full((n,), 0xEE, dtype=torch.uint8).pin_memory()
    for rep in range(2):
        k = fp.parse_f64_host_into(h_text, h_out, h_st)
        assert k == rb.size, rep
        assert np.array_equal(h_out[:k].numpy().view(np.uint64), rb), rep
        assert np.array_equal(h_st[:k].numpy(), rs), rep
        assert (h_st[k:k + 1000].numpy() == 0xEE).all()
    assert fp.get_error() == 0


def test_integer_file():
    """The integer file's shape (Section 12), alone and mixed with the bulk
    shapes: signs, leading zeros, values around 2^53 and up to 19 digits."""
    lines = workloads.integer_lines(2_000_000, 131)
    assert_parity("\n".join(lines).encode(), lines=lines)
    mixed = workloads.integer_lines(300_000, 132) + workloads.bulk_mixed_lines(100_000, 133)
    random.Random(134).shuffle(mixed)
    assert_parity("\n".join(mixed).encode(), lines=mixed)
