"""The oracle's C code under the compiler's sanitizers: AddressSanitizer and
UndefinedBehaviorSanitizer on hard cases, bulk fields, hexadecimal floats,
random and malformed strings and a 200 kB field (every field also parsed
alone from an exact-size copy), and ThreadSanitizer on its multi-threaded
buffer parse.  The driver is tests/native/oracle_sanitize.c."""
import os
import random
import shutil
import subprocess

import pytest

from paper_2101_11408_gb300 import workloads
from test_oracle_pins import _random_strings

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_C = os.path.join(os.path.dirname(HERE), "oracle", "oracle.c")
DRIVER = os.path.join(HERE, "native", "oracle_sanitize.c")


def _inputs(scale: int, huge: bool = True) -> bytes:
    rnd = random.Random(31)
    fuzz = ["".join(rnd.choice("0123456789" * 3 + "..eE+-  \t\r0xpP") for _ in range(rnd.randrange(32)))
            for _ in range(2000 * scale)]
    parts = [workloads.hard_case_text(300 * scale, 32), workloads.bulk_mixed_text(500 * scale, 33),
             workloads.hex_float_text(300 * scale, 34),
             "\n".join(_random_strings(rnd, 2000 * scale)).encode(), "\n".join(fuzz).encode(),
             b"", b"\n\n,,", b"0x1p-1075", b".e1", b"-", b"0x", b"1e", b"1e+"]
    if huge:
        parts += [b"1." + b"0" * 200000 + b"1", b"9" * 5000 + b"e-5000"]
    return b"\n".join(parts)


def _build_and_run(tmp_path, flags, data, timeout, args=()):
    cc = shutil.which("gcc")
    if not cc:
        pytest.skip("no gcc")
    exe = str(tmp_path / "oracle_sanitize")
    r = subprocess.run([cc, "-O1", "-g", "-std=gnu11", "-pthread"] + flags +
                       ["-o", exe, DRIVER, ORACLE_C], capture_output=True, text=True)
    if r.returncode:
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1",
               TSAN_OPTIONS="halt_on_error=1")
    r = subprocess.run([exe, *args], input=data, capture_output=True, timeout=timeout, env=env)
    out = r.stdout.decode() + r.stderr.decode()
    assert r.returncode == 0 and out.startswith("ok "), out[-3000:]
    assert "runtime error" not in out and "Sanitizer" not in out, out[-3000:]


def test_oracle_under_address_and_undefined_sanitizers(tmp_path):
    _build_and_run(tmp_path, ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined"],
                   _inputs(4), 600)


def test_oracle_buffer_parse_under_thread_sanitizer(tmp_path):
    _build_and_run(tmp_path, ["-fsanitize=thread"], _inputs(1, huge=False), 600, ["buffer"])
