"""The parse kernel on the CPU: fp_parse_kernel.cuh as it is, compiled for
the host with its PTX helpers replaced (tests/native/host_sync_stub.h) and
run as 1 to 4 blocks of 256 emulated threads (tests/native/parse_block_emu.cpp:
coroutines released warp by warp at each warp intrinsic and block by block
at each __syncthreads).  Counting, listing, staging, the look-back (over the
block's own earlier chunks and, with several blocks, other blocks'), the
tokenizers, Algorithm 1 and the stores must
give the oracle's count and every decided field's bits and status; the
fields left pending carry the queued status."""
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2101_11408_gb300 import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2101_11408_gb300", "csrc")
ST_PENDING_QUEUED = 0xFE


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("pbemu")
    with open(os.path.join(CSRC, "fp_parse_kernel.cuh")) as f:
        src = f.read()
    decl = "extern __shared__ __align__(128) uint8_t smem[];"
    assert src.count("#include <cuda_runtime.h>\n") == 1 and src.count(decl) == 1
    src = src.replace("#include <cuda_runtime.h>\n", "")
    src = src.replace(decl, "uint8_t* const smem = emu_block_smem();  // this block's buffer")
    (d / "fp_parse_kernel_host.cuh").write_text(src)
    shutil.copy(os.path.join(HERE, "native", "host_sync_stub.h"), d / "fp_sync.cuh")
    exe = str(d / "parse_block_emu")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Wno-unknown-pragmas",
                    "-Wno-unused-function", "-I", str(d), "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "native", "parse_block_emu.cpp")], check=True)
    return exe


def _check(exe, text: bytes, f32=False, grammar=0, chunk=16384, offset=0, max_pending=None,
           blocks=1, columns=0, rows_cap=0):
    extra = [str(columns), str(rows_cap)] if columns else []
    r = subprocess.run([exe, "32" if f32 else "64", str(grammar), str(chunk), str(offset),
                        str(blocks)] + extra, input=text, capture_output=True, timeout=600)
    out = r.stdout.decode().split("\n")[:-1]
    assert r.returncode == 0, out[-1:] + [r.stderr.decode()[-800:]]
    assert out[-1].startswith("count ")
    n = int(out[-1].split()[1])
    rb, rs = oracle.parse_buffer(text, b"," if columns else b"\n", f32=f32, grammar=grammar)
    assert n == rb.size, (n, rb.size)
    pending = 0
    for i in range(n):
        b, s = out[i].split()
        s = int(s)
        if s == ST_PENDING_QUEUED:
            pending += 1
            continue
        assert (int(b, 16), s) == (int(rb[i]), int(rs[i])), \
            (i, out[i], hex(int(rb[i])), int(rs[i]))
    if max_pending is not None:
        assert pending <= max_pending, pending
    return n, pending


@pytest.mark.parametrize("offset", [0, 3, 15])
def test_bulk_fields_across_many_chunks(emu, offset):
    # 20,000 numbers, about 376 kB: 23 chunks of 16 KiB, fields across their edges
    _check(emu, workloads.bulk_mixed_text(20000, workloads.SEED_BASE + 95), offset=offset,
           max_pending=0)


def test_small_chunks_and_binary32(emu):
    text = workloads.bulk_mixed_text(6000, workloads.SEED_BASE + 96)
    _check(emu, text, chunk=4096, offset=7, max_pending=0)
    _check(emu, text, f32=True, offset=1, max_pending=0)


def test_dense_chunks_listed_window_by_window(emu):
    """Short fields: more than 1024 starts per 16 KiB chunk, so the starts
    are listed window by window at parse time."""
    rnd = random.Random(97)
    lines = [rnd.choice(["1", "-0", "7e3", "", "9", "0.5", "x", "12"]) for _ in range(30000)]
    _check(emu, "\n".join(lines).encode(), offset=5, max_pending=0)


def test_grammar_edges_blanks_and_empty_fields(emu):
    from test_oracle_pins import _random_strings
    rnd = random.Random(98)
    lines = _random_strings(rnd, 4000)
    lines = [(" " * rnd.randrange(3)) + s + ("\t" if rnd.random() < 0.1 else "") for s in lines]
    lines += ["", "", " ", "\r", "+", "-", ".", "e5", "1e", "0x1p3", "1" * 70]
    text = "\n".join(lines).encode()
    _check(emu, text, offset=9)
    _check(emu, text + b"\n", offset=2)  # a final separator: no trailing empty field
    _check(emu, b"", offset=0)
    _check(emu, b"\n\n\n", offset=4)
    _check(emu, b"3.25", offset=11)


def test_hex_grammar_and_a_long_field(emu):
    """The hexadecimal mode: float.hex() values (the hexadecimal window
    tokenizer), decimal fields among them (the decimal one), and random
    hexadecimal shapes, some beyond the window (the general tokenizer)."""
    lines = workloads.hex_float_lines(3000, 99) + ["1.5", "2e-3", "0x1p-1075"]
    _check(emu, "\n".join(lines).encode(), grammar=1, offset=6, max_pending=0)
    rnd = random.Random(98)
    mixed = []
    for _ in range(4000):
        m = "".join(rnd.choice("0123456789abcdefABCDEF") for _ in range(rnd.randrange(1, 20)))
        if rnd.random() < 0.5:
            p = rnd.randrange(0, len(m) + 1)
            m = m[:p] + "." + m[p:]
        f = rnd.choice(["", "-", "+"]) + rnd.choice(["0x", "0X"]) + m
        if rnd.random() < 0.8:
            f += rnd.choice("pP") + rnd.choice(["", "+", "-"]) + str(rnd.randrange(0, 1100))
        mixed.append(f if rnd.random() < 0.9 else "%.17g" % rnd.random())
    _check(emu, "\n".join(mixed).encode(), grammar=1, offset=3, max_pending=0, blocks=2)
    big = b"1." + b"0" * 40000 + b"1"  # one field over several chunks: the fallback's
    n, pending = _check(emu, b"2.5\n" + big + b"\n-7", offset=0)
    assert n == 3 and pending == 1


def test_hard_cases_leave_long_fields_pending(emu):
    n, pending = _check(emu, workloads.hard_case_text(2000, workloads.SEED_BASE + 100), offset=13)
    assert 0 < pending < n


@pytest.mark.parametrize("blocks,chunk", [(2, 16384), (3, 4096), (4, 4096)])
def test_several_blocks_look_back_across_blocks(emu, blocks, chunk):
    """Blocks take chunk tickets in turn, so each chunk's prefix comes from
    other blocks' look-back words (aggregates and inclusive prefixes)."""
    text = workloads.bulk_mixed_text(25000, workloads.SEED_BASE + 101)
    _check(emu, text, chunk=chunk, offset=blocks, max_pending=0, blocks=blocks)
    rnd = random.Random(blocks)
    dense = "\n".join(rnd.choice(["1", "", "2.5", "x", "-3e2"]) for _ in range(40000)).encode()
    _check(emu, dense, chunk=chunk, offset=1, blocks=blocks, max_pending=0)


def test_json_mode(emu):
    """The kernel's JSON mode (its fast-path check of the JSON number rules)."""
    rnd = random.Random(102)
    lines = workloads.bulk_mixed_lines(6000, 103) + [
        rnd.choice(["+1", "01", "1.", ".5", "-0", "0.0", "1e5", "-1.5E-3", "00", "0e0", "-", "1.e2"])
        for _ in range(3000)]
    rnd.shuffle(lines)
    _check(emu, "\n".join(lines).encode(), grammar=2, offset=4, max_pending=0, blocks=2)


def test_column_major_mode(emu):
    """The column-major mode on well-formed rows: field i at column i mod 8,
    row i div 8 (a row's last field ends at '\n', the others at ',').
    Rows of the wrong shape (BAD_SHAPE) are the GPU tests' part."""
    text = workloads.csv_columns_text(3000, 8, 104)
    _check(emu, text, grammar=0, offset=8, columns=8, rows_cap=3000, max_pending=0, blocks=2)


def test_whole_path_on_the_hard_mix(emu, tmp_path):
    """Both kernels' code end to end on the CPU: the emulated parse kernel
    decides what it can and queues the rest (their statuses say so); the
    fallback kernel's per-field code, emulated, decides each queued field.
    Together every field of the hard-case mix equals the oracle."""
    from test_fallback_emulated import _body
    d = tmp_path / "fb"
    d.mkdir()
    (d / "fallback_body.inc").write_text(_body())
    fb = str(d / "fallback_emu")
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wno-unknown-pragmas", "-Wno-unused-function",
                    "-I", str(d), "-I", CSRC, "-o", fb,
                    os.path.join(HERE, "native", "fallback_emu.cpp")], check=True)
    lines = workloads.hard_case_lines(1500, workloads.SEED_BASE + 105)
    text = "\n".join(lines).encode()
    r = subprocess.run([emu, "64", "0", "16384", "5", "2"], input=text, capture_output=True,
                       timeout=600, check=True)
    out = r.stdout.decode().split("\n")[:-2]  # without the count line
    assert len(out) == len(lines)
    results = [tuple(int(x, 16) if j == 0 else int(x) for j, x in enumerate(ln.split()))
               for ln in out]
    queued = [i for i, (_, s) in enumerate(results) if s == ST_PENDING_QUEUED]
    assert queued
    r = subprocess.run([fb, "64", "0"], input="\n".join(lines[i] for i in queued).encode(),
                       capture_output=True, timeout=600, check=True)
    for i, ln in zip(queued, r.stdout.decode().split("\n")):
        b, s = ln.split()
        results[i] = (int(b, 16), int(s))
    rb, rs = oracle.parse_buffer(text)
    assert [(int(b), int(s)) for b, s in zip(rb, rs)] == results


@pytest.mark.parametrize("f32", [False, True])
def test_integer_groups(emu, f32):
    """Integer files (Section 12's integer set), alone and mixed with the
    bulk shapes: the oracle's results."""
    text = workloads.integer_text(6000, 123)
    _check(emu, text, f32=f32, max_pending=0)
    mixed = "\n".join(workloads.integer_lines(2000, 124) + workloads.bulk_mixed_lines(500, 125))
    _check(emu, mixed.encode(), f32=f32, max_pending=0)
