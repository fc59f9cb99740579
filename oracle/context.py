"""The C library's strtod on a delimited buffer, on host threads: a timing
context for the CPU baseline (the paper compares its method with the C
library's conversion).  Not the oracle and not a checker -- nothing is
compared with its results; only bench.py's CPU-baseline leg uses it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "strtod_context.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libstrtod_context.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile strtod_context.c (gcc, -O2, no arch flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra",
                    "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.context_strtod_buffer.argtypes = [
                ctypes.c_char_p, ctypes.c_size_t, ctypes.c_char, ctypes.c_int,
                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]
            lib.context_strtod_buffer.restype = ctypes.c_int
            _lib = lib
    return _lib


def strtod_buffer(text: bytes, delim: bytes = b"\n", threads: int | None = None) -> tuple[int, float]:
    """Convert every field of `text` with strtod on `threads` threads;
    returns (fields, seconds spent converting)."""
    n = ctypes.c_uint64()
    sec = ctypes.c_double()
    if _load().context_strtod_buffer(text, len(text), delim, threads or os.cpu_count() or 1,
                                     ctypes.byref(n), ctypes.byref(sec)):
        raise MemoryError("strtod context ran out of memory")
    return n.value, sec.value
