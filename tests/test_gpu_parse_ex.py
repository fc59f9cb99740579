"""fp_parse_ex on the GPU against the oracle: the JSON number grammar, the
hexadecimal-float grammar (short fields in the parse kernel, long ones in
the fallback kernel), and the column-major CSV layout with its shape rule,
in both formats, bit for bit."""
import random

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import workloads
from test_gpu_parity import join, to_device
from test_oracle_grammar_pins import JSON_INVALID, JSON_VALID, random_hex

pytestmark = pytest.mark.gpu
GRAMMAR = {"decimal": oracle.GRAMMAR_DEFAULT, "hex": oracle.GRAMMAR_HEX,
           "json": oracle.GRAMMAR_JSON}


def check(text, grammar="decimal", f32=False, delim=b"\n", offset=0, lines=None):
    t = to_device(text, offset)
    vals, st = fp.parse_ex(t, delim, f32=f32, grammar=grammar)
    torch.cuda.synchronize()
    assert fp.get_error() == 0
    got = vals.cpu().numpy().view(np.uint32 if f32 else np.uint64)
    gst = st.cpu().numpy()
    rb, rs = oracle.parse_buffer(text, delim, f32=f32, grammar=GRAMMAR[grammar])
    assert got.size == rb.size
    bad = np.nonzero((got != rb) | (gst != rs))[0]
    if bad.size:
        i = int(bad[0])
        what = lines[i][:80] if lines else "?"
        pytest.fail("%d mismatches; first at field %d %r: gpu %#x/%d oracle %#x/%d" % (
            bad.size, i, what, int(got[i]), int(gst[i]), int(rb[i]), int(rs[i])))


def json_lines(seed, n):
    rnd = random.Random(seed)
    lines = []
    for _ in range(n):
        k = rnd.randrange(4)
        if k == 0:
            lines.append(rnd.choice(JSON_VALID + JSON_INVALID))
        else:
            s = rnd.choice(["", "-", "+"]) + "".join(rnd.choice("0123456789")
                                                     for _ in range(rnd.randrange(0, 5)))
            if rnd.random() < 0.6:
                s += "." + "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(0, 4)))
            if rnd.random() < 0.4:
                s += rnd.choice("eE") + rnd.choice(["", "+", "-"]) + \
                    "".join(rnd.choice("0123456789") for _ in range(rnd.randrange(0, 4)))
            lines.append(s)
    return lines


@pytest.mark.parametrize("f32", [False, True])
def test_json_grammar(f32):
    lines = [x for x in json_lines(1, 60000) if "\n" not in x]
    check(join(lines), "json", f32, lines=lines)
    check(workloads.bulk_mixed_text(300000, 2), "json", f32)   # '+' and other forms: none here
    lines = workloads.hard_case_lines(5000, 3)                  # long fields: the fallback's JSON rules
    check(join(lines), "json", f32, lines=lines)


@pytest.mark.parametrize("f32", [False, True])
def test_hex_grammar(f32):
    rnd = random.Random(4)
    lines = [random_hex(rnd) for _ in range(50000)]
    lines += ["0x" + "f" * n + "p-%d" % rnd.randrange(0, 1200) for n in range(1, 200, 7)]  # long
    lines += ["0x1.8", "-0x0p0", "0x1p-1075", "0x1.8p-1074", "0x", "0xp3", "1.5", "1e5", "x"]
    check(join(lines), "hex", f32, lines=lines)
    check(workloads.bulk_mixed_text(200000, 5), "hex", f32)     # decimal fields still parse


@pytest.mark.parametrize("f32", [False, True])
def test_hex_workload_takes_the_hex_window(f32):
    """float.hex() values (the hexadecimal-float workload's recipe): every
    field decided in the parse kernel's hexadecimal mode by the hexadecimal
    window tokenizer (none reaches the general tokenizer), bit-exact with the
    oracle; then the same values as 4-column CSV rows (the hexadecimal and
    column-major modes together)."""
    n = 300000
    text = workloads.hex_float_text(n, workloads.SEED_BASE + 84)
    torch.cuda.synchronize()
    fp.stats(reset=True)
    check(text, "hex", f32)
    s = fp.stats(reset=True)
    assert s["fields"] == n and s["general_tokenizer"] == 0, s
    K = 4
    lines = text.split(b"\n")[:40000]
    csv = b"\n".join(b",".join(lines[r * K:(r + 1) * K]) for r in range(len(lines) // K))
    rows_cap = len(lines) // K + 2
    vals, st, cnt = fp.parse_ex(to_device(csv, 5), b",", f32=f32, grammar="hex", columns=K,
                                rows_cap=rows_cap)
    torch.cuda.synchronize()
    assert fp.get_error() == 0 and cnt == len(lines) // K * K
    rb, rs = oracle.parse_buffer(csv, b",", f32=f32, grammar=oracle.GRAMMAR_HEX)
    ov, ost = oracle.columnar(csv, rb, rs, K, rows_cap, b",")
    got = vals.cpu().numpy().reshape(-1).view(np.uint32 if f32 else np.uint64)
    gst = st.cpu().numpy().reshape(-1)
    filled = ost != 0xEE
    assert np.array_equal(gst, ost) and np.array_equal(got[filled], ov[filled])


def test_hex_and_json_are_off_by_default():
    lines = ["0x1p3", "+1", "01", ".5"]
    check(join(lines), "decimal", lines=lines)


def csv_block(rows, cols, seed, ragged=0.0, hard=0.0):
    rnd = random.Random(seed)
    vals = workloads.uniform_lines(rows * cols, seed)
    hard_vals = workloads.hard_case_lines(max(1, int(rows * cols * hard) + 1), seed + 1)
    out = []
    for r in range(rows):
        row = vals[r * cols:(r + 1) * cols]
        if hard:
            row = [rnd.choice(hard_vals) if rnd.random() < hard else v for v in row]
        if ragged and rnd.random() < ragged:
            row = row[:rnd.randrange(1, cols)] if rnd.random() < 0.5 else row + ["1.5"]
        out.append(",".join(row))
    return "\n".join(out).encode()


@pytest.mark.parametrize("f32", [False, True])
@pytest.mark.parametrize("shape", ["regular", "ragged", "hard"])
def test_columnar_layout(f32, shape):
    K = 8
    text = csv_block(20000, K, 6, ragged=0.01 if shape == "ragged" else 0.0,
                     hard=0.05 if shape == "hard" else 0.0)
    n_fields = oracle.count_fields(text, b",")
    rows_cap = (n_fields + K - 1) // K + 3
    t = to_device(text, 3)
    vals, st, n = fp.parse_ex(t, b",", f32=f32, columns=K, rows_cap=rows_cap)
    torch.cuda.synchronize()
    assert fp.get_error() == 0 and n == n_fields
    rb, rs = oracle.parse_buffer(text, b",", f32=f32)
    ov, ost = oracle.columnar(text, rb, rs, K, rows_cap, b",")
    got = vals.cpu().numpy().reshape(-1).view(np.uint32 if f32 else np.uint64)
    gst = st.cpu().numpy().reshape(-1)
    filled = ost != 0xEE
    assert np.array_equal(gst, ost)
    assert np.array_equal(got[filled], ov[filled])
    if shape == "regular":
        assert not (gst == oracle.STATUS_BAD_SHAPE).any()
    if shape == "ragged":
        assert (gst == oracle.STATUS_BAD_SHAPE).any()


def test_columnar_rows_cap_and_queue_overflow():
    """Fields beyond rows_cap are not stored; pending fields found by the
    overflow scan land in their column slots."""
    before = fp.get_config()
    try:
        fp.set_config(fallback_queue=1024, chunk_bytes=4096)  # runs with 8 KiB chunks
        K = 4
        text = csv_block(6000, K, 7, hard=0.5)
        n_fields = oracle.count_fields(text, b",")
        rows_cap = (n_fields + K - 1) // K
        t = to_device(text)
        fp.stats(reset=True)
        vals, st, n = fp.parse_ex(t, b",", columns=K, rows_cap=rows_cap)
        torch.cuda.synchronize()
        assert fp.stats()["queue_overflow"] > 0
        rb, rs = oracle.parse_buffer(text, b",")
        ov, ost = oracle.columnar(text, rb, rs, K, rows_cap, b",")
        filled = ost != 0xEE
        assert np.array_equal(st.cpu().numpy().reshape(-1), ost)
        assert np.array_equal(vals.cpu().numpy().reshape(-1).view(np.uint64)[filled], ov[filled])
        # a smaller rows_cap: the first rows are the same, the rest unwritten
        small = rows_cap // 2
        vals2, st2, n2 = fp.parse_ex(t, b",", columns=K, rows_cap=small)
        torch.cuda.synchronize()
        assert n2 == n_fields
        assert np.array_equal(st2.cpu().numpy()[:, :small], ost.reshape(K, rows_cap)[:, :small])
    finally:
        fp.set_config(**before)


def test_bad_options_are_refused():
    t = to_device(b"1,2\n3,4")
    for kw in (dict(columns=1, rows_cap=4), dict(columns=2, rows_cap=0)):
        with pytest.raises(fp._lib.FpError):
            fp.parse_ex(t, b",", **kw)
