"""The fallback kernel's per-field code on the CPU: warp_field and its
base-10^9 big-number helpers, taken from fp_fallback_kernel.cu as they are
and run by tests/native/fallback_emu.cpp with the 32 lanes of a warp as
lockstep coroutines (each warp intrinsic a rendezvous of all 32).  The
fallback kernel decides any field it is given, so every field of the
inputs -- long digit strings, exact midpoints, malformed long fields, short
fields of every shape -- must get the oracle's bits and status."""
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


def _body() -> str:
    """The kernel file's helpers and warp_field: from the anonymous namespace
    up to (not including) the per-item driver and the kernel."""
    with open(os.path.join(CSRC, "fp_fallback_kernel.cu")) as f:
        src = f.read()
    start = src.index("namespace {\n", src.index("namespace fp {")) + len("namespace {\n")
    end = src.index("// Decide pending field oi")
    return src[start:end]


@pytest.fixture(scope="module")
def emu(tmp_path_factory):
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("fbemu")
    (d / "fallback_body.inc").write_text(_body())
    exe = str(d / "fallback_emu")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Wno-unknown-pragmas",
                    "-Wno-unused-function", "-I", str(d), "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "native", "fallback_emu.cpp")], check=True)
    return exe


def _check(exe, lines, f32=False, grammar=0):
    text = "\n".join(lines).encode()
    r = subprocess.run([exe, "32" if f32 else "64", str(grammar)], input=text,
                       capture_output=True, timeout=900)
    out = r.stdout.decode().split("\n")[:-1]
    assert r.returncode == 0, (out[-1:] if out else "") + [r.stderr.decode()[-500:]]
    rb, rs = oracle.parse_buffer(text, f32=f32, grammar=grammar)
    assert len(out) == rb.size
    for i, ln in enumerate(out):
        b, s = ln.split()
        assert (int(b, 16), int(s)) == (int(rb[i]), int(rs[i])), \
            (lines[i][:90], ln, hex(int(rb[i])), int(rs[i]))


def test_hard_cases(emu):
    _check(emu, workloads.hard_case_lines(1500, workloads.SEED_BASE + 91))


def test_long_malformed_and_json(emu):
    from test_gpu_parity import _long_defects
    lines = _long_defects(random.Random(92), 1500)
    _check(emu, lines)
    _check(emu, lines[:800], grammar=2)


def test_short_fields_and_binary32(emu):
    from test_oracle_pins import _random_strings
    rnd = random.Random(93)
    lines = _random_strings(rnd, 1500) + ["", " ", "-0", "1e-400", "1e400", "0x1.8p3", ".5",
                                          "1.", "+.e1", "9" * 800 + "e-800"]
    _check(emu, lines)
    _check(emu, lines, f32=True)
    _check(emu, ["0x1.fffffep127", "0x1p-150", "-0X.8P1", "0x1.8p3"] + lines[:300], grammar=1)


def test_beyond_800_digits(emu):
    """Fields of more than 800 significant digits, where the fallback keeps
    800 and a sticky digit: exact midpoints padded with zeros (still ties)
    and with a nonzero digit far beyond (just above the midpoint)."""
    rng = np.random.Generator(np.random.PCG64(94))
    lines = []
    for b in rng.integers(1, 0x0010000000000000, size=120, dtype=np.int64).tolist():
        d, e = workloads.midpoint_decimal(int(b))  # subnormal midpoints: long expansions
        pad = max(0, 820 - len(d))
        lines.append("%s%se%d" % (d, "0" * pad, e - pad))
        lines.append("%s%s1e%d" % (d, "0" * pad, e - pad - 1))
        lines.append("%s%s9e%d" % (str(int(d) - 1), "9" * pad, e - pad - 1))
    _check(emu, lines)
