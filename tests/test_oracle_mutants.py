"""The pins are strong enough to catch a plausible slip in the oracle: each
mistake below is planted in a copy of oracle/oracle.c, built on the CPU,
and must disagree with CPython's correctly rounded float() on a fixed set
of fields (the paper's worked inputs, ties, subnormals, the overflow edge,
%.17g round trips), where the unmodified oracle agrees on every one."""
import ctypes
import os
import random
import shutil
import struct
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_C = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = [
    ("ties rounded up", "if (c > 0 || (c == 0 && (Q & 1))) Q += 1;",
     "if (c > 0 || (c == 0)) Q += 1;"),
    ("last place's exponent off by one", "int64_t e = (k > f->emin ? k : f->emin) - pm1;",
     "int64_t e = (k > f->emin ? k : f->emin) - f->p;"),
    ("overflow one binade early", "if (e > f->emax - pm1) {", "if (e >= f->emax - pm1) {"),
    ("subnormal cut", "} else if (Q < ((uint64_t)1 << pm1)) {",
     "} else if (Q <= ((uint64_t)1 << pm1)) {"),
    ("exponent sign dropped", "    *out = eneg ? -e : e;", "    *out = e;"),
]


def _fields():
    out = []
    with open(os.path.join(ROOT, "tests", "golden", "paper_examples.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                s = line.split("\t")[0]
                if not s.lower().startswith(("0x", "-0x")):
                    out.append(s)
    out += ["2.2250738585072011e-308", "2.2250738585072014e-308", "4.9406564584124654e-324",
            "2.4703282292062328e-324", "2.4703282292062327e-324", "1.7976931348623157e308",
            "1.7976931348623158e308", "1.7976931348623159e308", "123.456e-5", "5e-320"]
    rnd = random.Random(55)
    for _ in range(3000):
        x = struct.unpack("<d", struct.pack("<Q", rnd.getrandbits(63)))[0]
        if x == x and x not in (float("inf"),):
            out.append("%.17g" % x)
    return out


FIELDS = _fields()
TRUTH = [struct.unpack("<Q", struct.pack("<d", float(s)))[0] for s in FIELDS]


def _build(tmp_path, name, src):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no gcc")
    c = tmp_path / (name + ".c")
    c.write_text(src)
    so = str(tmp_path / (name + ".so"))
    subprocess.run([cc, "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", so, str(c)],
                   check=True)
    lib = ctypes.CDLL(so)
    lib.oracle_parse_field.argtypes = [ctypes.c_char_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_uint64),
                                       ctypes.POINTER(ctypes.c_uint8)]
    return lib


def _mismatches(lib):
    bits, st = ctypes.c_uint64(), ctypes.c_uint8()
    bad = 0
    for s, want in zip(FIELDS, TRUTH):
        b = s.encode()
        assert lib.oracle_parse_field(b, len(b), ctypes.byref(bits), ctypes.byref(st)) == 0
        bad += bits.value != want
    return bad


def test_unmodified_oracle_agrees(tmp_path):
    with open(ORACLE_C) as f:
        assert _mismatches(_build(tmp_path, "oracle", f.read())) == 0


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_slip_is_caught(tmp_path, what, old, new):
    with open(ORACLE_C) as f:
        src = f.read()
    assert src.count(old) == 1, what
    assert _mismatches(_build(tmp_path, "mutant", src.replace(old, new))) > 0, what
