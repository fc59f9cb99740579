"""Host-side checks of the C-ABI library: it loads, exports every symbol
include/*.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if h.endswith(".h"):
            with open(os.path.join(inc, h)) as f:
                names |= set(re.findall(r"FP_API [^;(]*?\b(fp_\w+)\s*\(", f.read()))
    return sorted(names)


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


def test_noalloc_refuses_sizes_before_any_cuda_call():
    # Only where no GPU is present: a refusal that regressed would reach the
    # CUDA calls, which then fail cleanly here (tests/test_zz_no_alloc.py
    # checks the same refusals on a GPU with real buffers behind the pointers).
    import torch
    if torch.cuda.is_available():
        pytest.skip("covered with real device buffers by the GPU tests")
    lib = _lib.load()
    cnt = ctypes.c_uint64()
    fake = ctypes.c_void_p(16)
    for n in ((1 << 64) - 9, 1 << 40):  # wraps in a chunk count; beyond 2^40
        assert lib.fp_parse_f64_noalloc(fake, n, b"\n", fake, fake, ctypes.addressof(cnt),
                                        None) == _lib.FP_ERR_ARG
    chunk = fp.get_config()["chunk_bytes"]
    assert lib.fp_parse_f64_noalloc(fake, 65536 * chunk + 1, b"\n", fake, fake,
                                    ctypes.addressof(cnt), None) == _lib.FP_ERR_CAPACITY
    assert lib.fp_parse_f64_noalloc(None, 10, b"\n", fake, fake, ctypes.addressof(cnt),
                                    None) == _lib.FP_ERR_ARG
    assert lib.fp_parse_f64_noalloc(fake, 10, b"\n", fake, fake, None, None) == _lib.FP_ERR_ARG


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


def test_struct_layouts_and_constants_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field
    offsets, and its constants the header's values: a C program built from
    include/fpparse.h (as C11) prints them."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"fp_stats_t": _lib.Stats, "fp_config_t": _lib.Config,
               "fp_server_config_t": _lib.ServerConfig, "fp_request_info_t": _lib.RequestInfo,
               "fp_server_stats_t": _lib.ServerStats, "fp_options_t": _lib.Options}
    consts = {"FP_OK": _lib.FP_OK, "FP_ERR_ARG": _lib.FP_ERR_ARG,
              "FP_ERR_CAPACITY": _lib.FP_ERR_CAPACITY, "FP_ERR_CUDA": _lib.FP_ERR_CUDA,
              "FP_ERR_BUDGET": _lib.FP_ERR_BUDGET, "FP_ERR_TIMEOUT": _lib.FP_ERR_TIMEOUT,
              "FP_ERR_INTERNAL": _lib.FP_ERR_INTERNAL, "FP_STATUS_OK": _lib.STATUS_OK,
              "FP_STATUS_INVALID": _lib.STATUS_INVALID, "FP_STATUS_OVERFLOW": _lib.STATUS_OVERFLOW,
              "FP_STATUS_UNDERFLOW": _lib.STATUS_UNDERFLOW,
              "FP_STATUS_BAD_SHAPE": _lib.STATUS_BAD_SHAPE, "FP_FORMAT_F64": _lib.FORMAT_F64,
              "FP_FORMAT_F32": _lib.FORMAT_F32, "FP_GRAMMAR_DECIMAL": _lib.GRAMMAR_DECIMAL,
              "FP_GRAMMAR_HEX": _lib.GRAMMAR_HEX, "FP_GRAMMAR_JSON": _lib.GRAMMAR_JSON}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fpparse.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    for name in consts:
        lines.append('  printf("%s %%lld\\n", (long long)%s);' % (name, name))
    lines += ["  return 0;", "}"]
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "abi")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, str(src)], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            *key, val = ln.split(" ")
            got[" ".join(key)] = int(val)
    for name, cls in structs.items():
        assert got[name + " size"] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got["%s %s" % (name, field)] == getattr(cls, field).offset, (name, field)
    for name, v in consts.items():
        assert got[name] == v, name


def test_c_program_links_and_calls_the_library(tmp_path):
    """A plain C program (tests/native/c_client.c) links against the
    library and gets the header's answers from the calls that need no GPU."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = _lib.library_path()
    exe = str(tmp_path / "c_client")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", exe, os.path.join(ROOT, "tests", "native", "c_client.c"),
                    lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
