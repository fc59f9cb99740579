"""fp_parse_f64_noalloc: the parse for callers that may not allocate memory
(fixed-memory or certified processes, plugins whose host owns every
allocation).  Its scratch is one fixed device array inside the library, so
its results must equal those of fp_parse_f64, which allocates per-stream
scratch, on consecutive calls whose inputs differ -- the array keeps each
call's contents, and the next call must not be affected by them.

This file is collected last on purpose; it also runs on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def _device_text(text: bytes) -> torch.Tensor:
    return torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()


def _run(entry, t: torch.Tensor):
    n = max(t.numel(), 1)
    out = torch.full((n,), -7.0, dtype=torch.float64, device=t.device)
    st = torch.full((n,), 0xEE, dtype=torch.uint8, device=t.device)
    cnt = torch.zeros(1, dtype=torch.int64, device=t.device)
    stream = torch.cuda.current_stream().cuda_stream
    rc = entry(t.data_ptr() if t.numel() else None, t.numel(), b"\n", out.data_ptr(),
               st.data_ptr(), cnt.data_ptr(), stream)
    assert rc == _lib.FP_OK, _lib.strerror(rc)
    torch.cuda.synchronize()
    k = int(cnt.item())
    return k, out[:k].cpu().numpy().view(np.uint64), st[:k].cpu().numpy()


def test_noalloc_matches_parse_f64_on_consecutive_calls():
    lib = _lib.load()
    inputs = [
        workloads.bulk_mixed_text(400_000, 901),   # larger first ...
        workloads.hard_case_text(20_000, 902),     # ... then another shape, using the fallback
        workloads.uniform_text(1000, 903),         # ... then a much smaller one
    ]
    for text in inputs:
        t = _device_text(text)
        ref = _run(lib.fp_parse_f64, t)
        got = _run(lib.fp_parse_f64_noalloc, t)
        assert got[0] == ref[0] and got[0] > 0
        assert np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2])
    # and once more with the first input, after the others left their state
    t = _device_text(inputs[0])
    assert np.array_equal(_run(lib.fp_parse_f64_noalloc, t)[1], _run(lib.fp_parse_f64, t)[1])


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    lib = _lib.load()
    chunk = fp.get_config()["chunk_bytes"]
    too_long = 65536 * chunk + 16
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    # nothing is read or written: the size is refused before any work is queued
    rc = lib.fp_parse_f64_noalloc(ctypes.c_void_p(16), too_long, b"\n", ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), cnt.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.FP_ERR_CAPACITY
