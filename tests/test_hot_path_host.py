"""The parse kernel's per-field arithmetic on the CPU: the device header's
window tokenizer (Section 4), Algorithm 1 (Section 5) and the general
tokenizer with the 19-digit check (Section 11), built for the host
(tests/native/hot_path_check.cpp), against the oracle on seeded fields.

Every field the two tokenizers decide must carry the oracle's bit pattern
and status; the rest are the fallback kernel's and are only counted (the
GPU parity tests cover them).  This catches a slip in the hot path's
arithmetic without a GPU; the kernel's indexing, staging and look-back are
the GPU tests' part.
"""
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


@pytest.fixture(scope="module")
def hot_path(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("hot") / "hot_path_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Wno-unknown-pragmas", "-I", CSRC,
                    "-o", exe, os.path.join(HERE, "native", "hot_path_check.cpp")], check=True)
    return exe


def run_hot_path(exe, text: bytes, f32=False, grammar=0, stderr=None):
    """Decided fields as (index, bits, status) arrays, and the pending count
    (the harness's report, "hex_window <fields>", goes into stderr if given)."""
    r = subprocess.run([exe, "32" if f32 else "64", str(grammar)], input=text,
                       capture_output=True, timeout=600, check=True)
    if stderr is not None:
        stderr.append(r.stderr.decode())
    lines = r.stdout.split(b"\n")[:-1]
    idx, bits, st = [], [], []
    pending = 0
    for i, ln in enumerate(lines):
        if ln == b"P":
            pending += 1
            continue
        b, s = ln.split()
        idx.append(i)
        bits.append(int(b, 16))
        st.append(int(s))
    return len(lines), np.array(idx, dtype=np.int64), np.array(bits, dtype=np.uint64), \
        np.array(st, dtype=np.uint8), pending


def check(exe, text: bytes, f32=False, grammar=0, max_pending=None, stderr=None):
    n, idx, bits, st, pending = run_hot_path(exe, text, f32, grammar, stderr)
    rb, rs = oracle.parse_buffer(text, f32=f32, grammar=grammar)
    assert n == rb.size, "field counts differ"
    want_b = rb.astype(np.uint64)[idx]
    want_s = rs[idx]
    bad = np.nonzero((want_b != bits) | (want_s != st))[0]
    if bad.size:
        fields = text.split(b"\n")
        k = int(idx[bad[0]])
        raise AssertionError("field %d %r: hot path %016x/%d, oracle %016x/%d (%d mismatches)"
                             % (k, fields[k], int(bits[bad[0]]), int(st[bad[0]]),
                                int(want_b[bad[0]]), int(want_s[bad[0]]), bad.size))
    if max_pending is not None:
        assert pending <= max_pending, "%d fields left to the fallback" % pending
    return n, pending


@pytest.mark.parametrize("f32", [False, True])
def test_bulk_mixed_fields(hot_path, f32):
    """The bulk workload's shapes (17-digit uniforms, coordinates, integers
    below 2^63, d.ddddE+-xxx): all decided on the hot path."""
    n, pending = check(hot_path, workloads.bulk_mixed_text(30000, workloads.SEED_BASE + 71), f32,
                       max_pending=0)
    assert n == 30000


def test_uniform_fields(hot_path):
    check(hot_path, workloads.uniform_text(20000, workloads.SEED_BASE + 72), max_pending=0)


@pytest.mark.parametrize("f32", [False, True])
def test_decimal_range_boundaries(hot_path, f32):
    """One- and two-digit significands at every exponent from 10^-345 to
    10^310: underflow to zero, subnormals, the normal range, overflow."""
    lines = []
    for d in list(range(1, 10)) + list(range(10, 100, 7)):
        for ex in range(-345, 311):
            lines.append("%de%d" % (d, ex))
            lines.append("-%d.%de%d" % (d // 10 or d, d % 10, ex))
    check(hot_path, "\n".join(lines).encode(), f32, max_pending=0)


def _fuzz_fields(count, seed, alphabet):
    rnd = random.Random(seed)
    out = []
    for _ in range(count):
        n = rnd.randrange(0, 32)
        out.append("".join(rnd.choice(alphabet) for _ in range(n)))
    return "\n".join(out).encode()


@pytest.mark.parametrize("grammar", [0, 2])
def test_grammar_fuzz(hot_path, grammar):
    """Short fields over digits, points, markers, signs and blanks: most
    are malformed, and the two tokenizers must classify every one as the
    oracle does (decimal and JSON grammars)."""
    alphabet = "0123456789" * 3 + "..eE+-  \t\r0x"
    text = _fuzz_fields(40000, 73 + grammar, alphabet)
    check(hot_path, text, grammar=grammar)


def test_digit_heavy_fuzz(hot_path):
    """Mostly digits with at most a point and an exponent: lengths around
    the 19-digit and 24-character limits of the window tokenizer."""
    rnd = random.Random(74)
    lines = []
    for _ in range(40000):
        nd = rnd.randrange(1, 27)
        digs = "".join(rnd.choice("0123456789") for _ in range(nd))
        if rnd.random() < 0.6:
            p = rnd.randrange(0, nd + 1)
            digs = digs[:p] + "." + digs[p:]
        if rnd.random() < 0.4:
            digs += rnd.choice("eE") + rnd.choice(["", "+", "-"]) + str(rnd.randrange(0, 400))
        if rnd.random() < 0.3:
            digs = rnd.choice("+-") + digs
        lines.append(digs)
    n, pending = check(hot_path, "\n".join(lines).encode())
    assert pending < n // 4


@pytest.mark.parametrize("f32", [False, True])
def test_hex_floats(hot_path, f32):
    """Hexadecimal floats (Appendix C's grammar option) and decimal fields
    under the hexadecimal grammar."""
    rnd = random.Random(75)
    lines = []
    for _ in range(20000):
        m = "".join(rnd.choice("0123456789abcdefABCDEF") for _ in range(rnd.randrange(1, 20)))
        if rnd.random() < 0.5:
            p = rnd.randrange(0, len(m) + 1)
            m = m[:p] + "." + m[p:]
        s = rnd.choice(["", "-", "+"]) + rnd.choice(["0x", "0X"]) + m
        if rnd.random() < 0.8:
            s += rnd.choice("pP") + rnd.choice(["", "+", "-"]) + str(rnd.randrange(0, 1100))
        lines.append(s)
    lines += ["1.5", "-0.25e-3", "0x", "0x.p1", "0x1p", "0x1g", "0X1P-1074", "0x1p-1075",
              "0x1.fffffffffffff8p1023", "0x1.fffffffffffff7p1023"]
    check(hot_path, "\n".join(lines).encode(), f32, grammar=1)


@pytest.mark.parametrize("f32", [False, True])
def test_hex_window_decides_the_hex_workload(hot_path, f32):
    """The hexadecimal-float workload (float.hex() of uniform values and of
    random finite bit patterns: subnormals, zeros, both signs, exponents to
    +-1023) plus hand-made shapes at the window's edges: every field of the
    workload is decided by the hexadecimal window tokenizer, bit-exact with
    the oracle (the value is dyadic: one rounding of the exact significand x
    2^exponent, Appendix C)."""
    text = workloads.hex_float_text(20000, workloads.SEED_BASE + 83)
    err = []
    n, _ = check(hot_path, text, f32, grammar=1, max_pending=0, stderr=err)
    assert err[-1].split() == ["hex_window", str(n)]
    edges = ["0x1p0", "0x.8p1", "0x1.p0", "0X1.8P3", "+0x1p-1", "-0x0p+0", "0x0.0p-9999",
             "0x1p+9999", "0x1p-1074", "0x1p-1075", "0x1.8p-1075", "0x1.fffffffffffffp+1023",
             "0x1.fffffffffffff8p+1023", "0xffffffffffffffffp0", "0x1ffffffffffffffffp0",
             "0x0000000000000001.0p0", "0x1.0000000000000000p0", "0xabcdefABCDEFp-20",
             "0x1.99999999999999999p-4", "0x1pp1", "0x1.8.p1", "0x1p1a", "0x1p+", "0xp1",
             "0x1.gp1", "0x1p12345", "-0x1.0000000000001p-1022", "0x123456789abcdefp-2",
             "0x1.8p1 ", " 0x1.8p1", "0x1.8", "0x1_8p1"]
    check(hot_path, "\n".join(edges).encode(), f32, grammar=1)


def test_hard_cases_decided_where_possible(hot_path):
    """The hard-case mix: long fields go to the fallback kernel; the short
    ones the hot path settles (17-25 digits near the range ends) must be
    exact."""
    n, pending = check(hot_path, workloads.hard_case_text(3000, workloads.SEED_BASE + 76))
    assert pending < n


def _exact_midpoints(count, seed):
    """Midpoints between adjacent doubles of magnitude 2^49 .. 2^63 (unit in
    the last place 2^-3 .. 2^10; below 10^19, so no 20-digit integers),
    written exactly in decimal with at most 19
    significant digits (so q lies in [-4, 23], the range of exact ties,
    Section 6), and each one's neighbours one unit away in its last digit."""
    import math
    from decimal import Decimal, getcontext
    getcontext().prec = 60
    rnd = random.Random(seed)
    out = []
    while len(out) < count:
        e = rnd.randrange(49, 63)
        x = float(rnd.randrange(1 << 52, 1 << 53)) * 2.0 ** (e - 52)
        h = Decimal(x) + Decimal(math.ulp(x)) / 2  # exact
        digits, exp = h.as_tuple().digits, h.as_tuple().exponent
        sig = "".join(map(str, digits)).rstrip("0")
        if len(sig) > 19:
            continue
        last = Decimal(1).scaleb(exp)
        for v in (h, h + last, h - last):
            s = format(v, "f")
            if "." not in s and rnd.random() < 0.5:  # trailing zeros as an exponent: q > 0
                t = s.rstrip("0")
                s = "%se%d" % (t, len(s) - len(t)) if len(t) < len(s) else s
            out.append(s)
    return out


@pytest.mark.parametrize("f32", [False, True])
def test_exact_ties_and_their_neighbours(hot_path, f32):
    """Ties go to the even significand (Algorithm 1's tie test, Sections 6,
    8.1 and 9.1); one unit above or below in the last digit goes to that
    side.  Half of them with a point, so q runs over [-4, 0] too."""
    lines = _exact_midpoints(6000, 77)
    lines += ["9007199254740993", "9007199254740995", "4503599627370496.5", "4503599627370497.5",
              "2251799813685248.25", "2251799813685248.75", "1125899906842624.125"]
    check(hot_path, "\n".join(lines).encode(), f32, max_pending=0)


def _top_of_tie_range_fields():
    """Ties at q = 23, the top of the exact-tie range (Section 6): 2^k 10^23
    has the 54-bit odd part 5^23, so it lies halfway between two doubles
    (10^23 itself is the classic case).  Written plainly they reach the
    window tokenizer with the exponent part as trailing zeros (q below 23);
    with blanks around them they reach the general tokenizer with q = 23.
    Their neighbours one unit away go to that side."""
    out = []
    for k in range(0, 14):
        for w in (2 ** k, 2 ** k + 1, 2 ** k - 1 if k else 3):
            for fmt in ("%de23", " %de23", "%de23 ", "\t%dE+23"):
                out.append(fmt % w)
    return out


@pytest.mark.parametrize("f32", [False, True])
def test_ties_at_the_top_of_the_tie_range(hot_path, f32):
    check(hot_path, "\n".join(_top_of_tie_range_fields()).encode(), f32, max_pending=0)


def test_word_wide_byte_tests():
    """The tokenizers' word-wide byte tests (tests/native/swar_check.cpp)
    against byte-by-byte definitions, on four million words."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "swar_check")
        subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Wno-unknown-pragmas", "-I", CSRC,
                        "-o", exe, os.path.join(HERE, "native", "swar_check.cpp")], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_hot_path_under_sanitizers(tmp_path):
    """The device header's per-field arithmetic, built for the host with
    AddressSanitizer and UndefinedBehaviorSanitizer: no read outside the
    padded tile, no oversized shift or signed overflow, on bulk fields, the
    grammar fuzz, exact ties, range boundaries and hexadecimal floats."""
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    exe = str(tmp_path / "hot_path_san")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-Wno-unknown-pragmas", "-I", CSRC,
                        "-o", exe, os.path.join(HERE, "native", "hot_path_check.cpp")],
                       capture_output=True, text=True)
    if r.returncode:
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
    texts = [workloads.bulk_mixed_text(10000, workloads.SEED_BASE + 78),
             _fuzz_fields(10000, 79, "0123456789" * 3 + "..eE+-  \t\r0x"),
             "\n".join(_exact_midpoints(1000, 80)).encode(),
             "\n".join("%de%d" % (d, e) for d in (1, 9, 47, 99) for e in range(-400, 400)).encode(),
             workloads.hex_float_text(3000, workloads.SEED_BASE + 82)]
    for t in texts:
        for fmt in ("64", "32"):
            for grammar in ("0", "1", "2"):
                r = subprocess.run([exe, fmt, grammar], input=t, capture_output=True, timeout=300)
                err = r.stderr.decode()
                assert r.returncode == 0 and "runtime error" not in err and "Sanitizer" not in err, \
                    err[:2000]


HOT_MUTANTS = [
    ("tie range", "static constexpr int TIE_QMIN = -4, TIE_QMAX = 23;",
     "static constexpr int TIE_QMIN = -4, TIE_QMAX = 22;"),
    ("point's exponent", "t.q = ex + (hp ? dpos - 23 : em - 24);",
     "t.q = ex + (hp ? dpos - 22 : em - 24);"),
    ("exponent part as zeros", "t.q = ex + (hp ? dpos - 23 : em - 24);",
     "t.q = ex + (hp ? dpos - 23 : em - 23);"),
    ("exponent's sign", "      if (ch == '-') ex = -ex;\n", ""),
    ("single point", "  if (Ms & (Ms - 1u)) return false;\n", ""),
    ("rounding step", "  m = (m + 1) >> 1;\n", "  m = m >> 1;\n"),
    ("overflow to infinity", "  r.bits = ovf ? F::INF : bits;\n", "  r.bits = bits;\n"),
    ("overflow status", "  r.status = ovf ? ST_OVERFLOW : ST_OK;\n", "  r.status = ST_OK;\n"),
    ("underflow status", "    r.status = m ? ST_OK : ST_UNDERFLOW;\n", "    r.status = ST_OK;\n"),
    ("19-digit truncation", "      exp_adj++;\n      sticky |= (d != 0);", "      sticky |= (d != 0);"),
    ("w+1 check", "    ElResult b = convert_wq<F>(w + 1, q, tab, true);",
     "    ElResult b = convert_wq<F>(w, q, tab, true);"),
    ("hex letter value", "hex4((x[j] & 0x0F0F0F0Fu) + 9u * ((x[j] >> 6) & 0x01010101u))",
     "hex4((x[j] & 0x0F0F0F0Fu) + 10u * ((x[j] >> 6) & 0x01010101u))"),
    ("hex fraction digits", "(int64_t)ex - 4 * (hp ? pp - 1 - dpos : 0)",
     "(int64_t)ex - 4 * (hp ? pp - dpos : 0)"),
    ("hex exponent part", "const uint32_t zs = 4u * (uint32_t)(24 - pp);",
     "const uint32_t zs = 4u * (uint32_t)(23 - pp);"),
    ("hex significand limit", "  if (v_hi >> zs) return false;", ""),
    ("hex single point", "  if (Mp & (Mp - 1u)) return false;\n", ""),
    ("JSON leading zero",
     "    ok = ok && nint > 0 && !(nint > 1 && s[int_start] == '0') && !(point && ndig == nint);",
     "    ok = ok && nint > 0 && !(point && ndig == nint);"),
]


@pytest.mark.parametrize("what,old,new", HOT_MUTANTS, ids=[m[0] for m in HOT_MUTANTS])
def test_planted_slip_in_the_hot_path_is_caught(tmp_path, what, old, new):
    """Each slip planted in a host copy of the device header fails one of the
    checks above (bulk fields, range boundaries, digit-heavy and grammar
    fuzz, exact ties, hard cases, ties at the top of the tie range)."""
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    d = tmp_path / "csrc"
    shutil.copytree(CSRC, d, ignore=shutil.ignore_patterns("*.o", "*.so", "_build"))
    hdr = d / "fp_device.cuh"
    src = hdr.read_text()
    assert src.count(old) == 1, what
    hdr.write_text(src.replace(old, new))
    exe = str(tmp_path / "hot_mutant")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wno-unknown-pragmas", "-I", str(d), "-o", exe,
                    os.path.join(HERE, "native", "hot_path_check.cpp")], check=True)
    checks = [lambda: check(exe, workloads.bulk_mixed_text(30000, workloads.SEED_BASE + 71)),
              lambda: test_decimal_range_boundaries(exe, False),
              lambda: test_digit_heavy_fuzz(exe),
              lambda: test_exact_ties_and_their_neighbours(exe, False),
              lambda: test_grammar_fuzz(exe, 2),
              lambda: test_hard_cases_decided_where_possible(exe),
              lambda: test_ties_at_the_top_of_the_tie_range(exe, False),
              lambda: test_hex_floats(exe, False),
              lambda: test_hex_window_decides_the_hex_workload(exe, False)]
    caught = 0
    for c in checks:
        try:
            c()
        except AssertionError:
            caught += 1
    assert caught > 0, what
