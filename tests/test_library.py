"""Host-side checks of the C-ABI library: it loads, exports every symbol
include/fpparse.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "fpparse.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"FP_API [^;(]*?\b(fp_\w+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a_only():
    from paper_2101_11408_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_max_fields():
    assert fp.max_fields(0) == 0
    assert fp.max_fields(1) == 1
    assert fp.max_fields(12345) == 12345


def test_argument_errors_need_no_gpu():
    lib = _lib.load()
    cnt = ctypes.c_uint64()
    # NULL text with len > 0
    assert lib.fp_parse_f64(None, 10, b"\n", None, None, ctypes.addressof(cnt), None) == \
        _lib.FP_ERR_ARG
    # NULL count
    assert lib.fp_parse_f64(None, 0, b"\n", None, None, None, None) == _lib.FP_ERR_ARG
    # length beyond 2^40
    assert lib.fp_parse_f64(ctypes.c_void_p(16), 1 << 40, b"\n", ctypes.c_void_p(16),
                            ctypes.c_void_p(16), ctypes.addressof(cnt), None) == _lib.FP_ERR_ARG
    # batch: zero buffers, decreasing offsets
    ptrs = (ctypes.c_void_p * 2)(16, 32)
    lens = (ctypes.c_size_t * 2)(4, 4)
    offs = (ctypes.c_uint64 * 3)(0, 8, 4)
    cnts = (ctypes.c_uint64 * 2)()
    assert lib.fp_parse_f64_batch(ptrs, lens, 0, b"\n", ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  offs, cnts, None) == _lib.FP_ERR_ARG
    assert lib.fp_parse_f64_batch(ptrs, lens, 2, b"\n", ctypes.c_void_p(16), ctypes.c_void_p(16),
                                  offs, cnts, None) == _lib.FP_ERR_ARG
    assert lib.fp_get_stats(None, 0, None) == _lib.FP_ERR_ARG


def test_config_validation():
    before = fp.get_config()
    with pytest.raises(fp.FpError):
        fp.set_config(chunk_bytes=5000)
    with pytest.raises(fp.FpError):
        fp.set_config(ctas_per_sm=9)
    with pytest.raises(fp.FpError):
        fp.set_config(fallback_queue=10)
    assert fp.get_config() == before
    c = fp.set_config(chunk_bytes=4096, ctas_per_sm=2)
    assert c["chunk_bytes"] == 4096 and c["ctas_per_sm"] == 2
    fp.set_config(**before)
    assert fp.get_config() == before


def test_strerror():
    assert _lib.strerror(0) == "ok"
    assert "argument" in _lib.strerror(1)


def test_python_api_rejects_host_tensors():
    import torch
    with pytest.raises(TypeError):
        fp.parse_f64(torch.zeros(4, dtype=torch.uint8))
    with pytest.raises(TypeError):
        fp.parse_f64(torch.zeros(4, dtype=torch.int32))


def test_host_entry_refuses_arrays_it_would_overrun():
    """parse_f64_host_into writes up to len(text) results through raw host
    addresses: arrays of another dtype, too short, non-contiguous or
    read-only are refused before the library is called."""
    import numpy as np
    import torch
    text = np.frombuffer(b"1.5\n2\n3\n", dtype=np.uint8)
    n = text.size
    ok_v, ok_s = np.empty(n, np.float64), np.empty(n, np.uint8)
    bad = [(np.empty(n - 1, np.float64), ok_s),
           (ok_v, np.empty(n - 1, np.uint8)),
           (np.empty(n, np.float32), ok_s),
           (np.empty(2 * n, np.float64)[::2], ok_s),
           (ok_v, np.frombuffer(bytes(n), dtype=np.uint8)),
           (torch.empty(n, dtype=torch.float32), ok_s),
           ([0.0] * n, ok_s)]
    for v, s in bad:
        with pytest.raises((TypeError, ValueError)):
            fp.parse_f64_host_into(text, v, s)
    with pytest.raises(TypeError):
        fp.parse_f64_host_into(text.astype(np.int8), ok_v, ok_s)
