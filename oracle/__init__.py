"""Exact CPU oracle for decimal text -> binary64 (and binary32) parsing.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the library under
``paper_2101_11408_gb300`` never does.  The arithmetic lives in ``oracle.c``
(plain C, exact big naturals); this module compiles it with gcc and calls it
through ctypes.

Functions follow the problem statement of the paper (Section 1: nearest
binary64, ties to even; Section 2: the binary64 and binary32 formats;
Section 4: the string grammar and its explicit bounds).  Parity status: the
binary64 functions are pinned by the paper's worked examples, by closed forms
(exact integers, exact powers of ten, constructed midpoints between adjacent
doubles) and by CPython's correctly rounded ``float()``
(``tests/test_oracle_pins.py``); the binary32 functions by float32 round
trips, constructed float32 midpoints, exact integers and powers of ten,
range boundaries and a neighbour-comparison brute force
(``tests/test_oracle_f32_pins.py``); the grammars and the columnar layout by
``tests/test_oracle_grammar_pins.py`` (the JSON number grammar's accepted
and rejected forms, CPython's correctly rounded ``float.fromhex`` on
hexadecimal floats, Appendix C's printed pairs, hand-checked layouts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

STATUS_OK, STATUS_INVALID, STATUS_OVERFLOW, STATUS_UNDERFLOW, STATUS_BAD_SHAPE = 0, 1, 2, 3, 4
GRAMMAR_DEFAULT, GRAMMAR_HEX, GRAMMAR_JSON = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, no arch flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
           "-Wall", "-Wextra", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_parse_field.argtypes = [
                ctypes.c_char_p, ctypes.c_size_t,
                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint8)]
            lib.oracle_parse_field.restype = ctypes.c_int
            lib.oracle_count_fields.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_char]
            lib.oracle_count_fields.restype = ctypes.c_uint64
            lib.oracle_parse_buffer.argtypes = [
                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_char,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
            lib.oracle_parse_buffer.restype = ctypes.c_int
            lib.oracle_parse_field_f32.argtypes = [
                ctypes.c_char_p, ctypes.c_size_t,
                ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint8)]
            lib.oracle_parse_field_f32.restype = ctypes.c_int
            lib.oracle_parse_buffer_f32.argtypes = lib.oracle_parse_buffer.argtypes
            lib.oracle_parse_buffer_f32.restype = ctypes.c_int
            lib.oracle_parse_field_ex.argtypes = [
                ctypes.c_char_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint8)]
            lib.oracle_parse_field_ex.restype = ctypes.c_int
            lib.oracle_parse_buffer_ex.argtypes = [
                ctypes.c_void_p, ctypes.c_size_t, ctypes.c_char, ctypes.c_int, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]
            lib.oracle_parse_buffer_ex.restype = ctypes.c_int
            _lib = lib
    return _lib


def parse_field(s) -> tuple[int, int]:
    """Parse one field; returns (binary64 bit pattern, status)."""
    if isinstance(s, str):
        s = s.encode("utf-8")
    lib = _load()
    bits = ctypes.c_uint64()
    st = ctypes.c_uint8()
    if lib.oracle_parse_field(s, len(s), ctypes.byref(bits), ctypes.byref(st)):
        raise MemoryError("oracle ran out of memory")
    return bits.value, st.value


def parse_field_f32(s) -> tuple[int, int]:
    """Parse one field to binary32; returns (bit pattern, status)."""
    if isinstance(s, str):
        s = s.encode("utf-8")
    lib = _load()
    bits = ctypes.c_uint32()
    st = ctypes.c_uint8()
    if lib.oracle_parse_field_f32(s, len(s), ctypes.byref(bits), ctypes.byref(st)):
        raise MemoryError("oracle ran out of memory")
    return bits.value, st.value


def parse_field_ex(s, f32: bool = False, grammar: int = GRAMMAR_DEFAULT) -> tuple[int, int]:
    """One field in either format under a grammar (GRAMMAR_DEFAULT, the
    decimal grammar; GRAMMAR_HEX, that or a hexadecimal float; GRAMMAR_JSON,
    the JSON number grammar).  Returns (bit pattern, status)."""
    if isinstance(s, str):
        s = s.encode("utf-8")
    lib = _load()
    bits = ctypes.c_uint64()
    st = ctypes.c_uint8()
    if lib.oracle_parse_field_ex(s, len(s), int(f32), int(grammar), ctypes.byref(bits),
                                 ctypes.byref(st)):
        raise MemoryError("oracle ran out of memory")
    return bits.value, st.value


def count_fields(text: bytes, delim: bytes = b"\n") -> int:
    lib = _load()
    buf = np.frombuffer(text, dtype=np.uint8)
    return int(lib.oracle_count_fields(buf.ctypes.data, len(text), delim))


def parse_buffer(text, delim: bytes = b"\n", nthreads: int | None = None, f32: bool = False,
                 grammar: int = GRAMMAR_DEFAULT):
    """Parse every field of a buffer.

    Returns (bits: uint64 array, status: uint8 array), or with f32=True
    (bits: uint32 array of binary32 patterns, status).  ``text`` is bytes or
    a uint8 numpy array.
    """
    lib = _load()
    if isinstance(text, (bytes, bytearray, memoryview)):
        buf = np.frombuffer(bytes(text), dtype=np.uint8)
    else:
        buf = np.ascontiguousarray(text, dtype=np.uint8)
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    n = int(lib.oracle_count_fields(buf.ctypes.data, buf.size, delim))
    bits = np.zeros(max(n, 1), dtype=np.uint32 if f32 else np.uint64)
    st = np.zeros(max(n, 1), dtype=np.uint8)
    cnt = ctypes.c_uint64()
    rc = lib.oracle_parse_buffer_ex(buf.ctypes.data, buf.size, delim, int(f32), int(grammar),
                                    bits.ctypes.data, st.ctypes.data, bits.size,
                                    ctypes.byref(cnt), int(nthreads))
    if rc:
        raise MemoryError("oracle failed (capacity or memory)")
    assert cnt.value == n
    return bits[:n], st[:n]


def columnar(text, bits, status, columns: int, rows_cap: int, delim: bytes = b","):
    """Column-major layout of row-order results (the fused CSV form): field i
    of the buffer goes to column i mod K, row i div K, i.e. entry
    (i mod K) * rows_cap + i div K.  A field whose terminator disagrees with
    its column -- the last column must end at '\n' or at the end of the
    buffer, every other column at `delim` -- gets STATUS_BAD_SHAPE (its value
    is kept).  Returns (values, statuses) of K * rows_cap entries; entries no
    field reaches are left as zero / 0xEE."""
    buf = np.frombuffer(bytes(text), dtype=np.uint8)
    n = bits.size
    k = np.arange(n)
    seps = np.nonzero((buf == ord("\n")) | (buf == ord(delim)))[0]
    term = np.full(n, ord("\n"), dtype=np.uint8)  # the buffer's end counts as '\n'
    m = min(n, seps.size)
    term[:m] = buf[seps[:m]]
    last_col = (k % columns) == columns - 1
    bad = (term == ord("\n")) != last_col
    st = status.copy()
    st[bad] = STATUS_BAD_SHAPE
    if n and (n - 1) // columns >= rows_cap:
        raise ValueError("rows_cap too small")
    out = np.zeros(columns * rows_cap, dtype=bits.dtype)
    ost = np.full(columns * rows_cap, 0xEE, dtype=np.uint8)
    dest = (k % columns) * rows_cap + k // columns
    out[dest] = bits
    ost[dest] = st
    return out, ost


def bits_to_float(bits: int) -> float:
    return np.array([bits], dtype=np.uint64).view(np.float64)[0].item()
