"""fp_parse_f64_noalloc: the parse for callers that may not allocate memory
once running (fixed-memory or certified processes, plugins whose host owns
every allocation).  Its scratch is one fixed device array inside the
library, kept between calls, so each call must give the oracle's results --
and the same results as fp_parse_f64, which allocates per-stream scratch --
whatever the previous call left in the array; once set up on a device it
must allocate nothing; and it must refuse sizes beyond the array with real
buffers in place, so that a regression in the check fails an assertion
instead of touching memory the call does not own.

This file is collected last on purpose; it also runs on its own.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

NOALLOC_QUEUE = 65536       # fallback queue entries of the fixed array
NOALLOC_MAX_CHUNKS = 65536  # chunks of the fixed array


def _device_text(text: bytes) -> torch.Tensor:
    return torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()


def _outputs(n: int, dev):
    n = max(n, 1)
    return (torch.full((n,), -7.0, dtype=torch.float64, device=dev),
            torch.full((n,), 0xEE, dtype=torch.uint8, device=dev),
            torch.zeros(1, dtype=torch.int64, device=dev))


def _call(entry, t: torch.Tensor, outs):
    out, st, cnt = outs
    stream = torch.cuda.current_stream().cuda_stream
    return entry(t.data_ptr() if t.numel() else None, t.numel(), b"\n", out.data_ptr(),
                 st.data_ptr(), cnt.data_ptr(), stream)


def _run(entry, t: torch.Tensor):
    outs = _outputs(t.numel(), t.device)
    rc = _call(entry, t, outs)
    assert rc == _lib.FP_OK, _lib.strerror(rc)
    torch.cuda.synchronize()
    out, st, cnt = outs
    k = int(cnt.item())
    return k, out[:k].cpu().numpy().view(np.uint64), st[:k].cpu().numpy()


def test_noalloc_matches_the_oracle_and_parse_f64_on_consecutive_calls():
    lib = _lib.load()
    inputs = [
        workloads.bulk_mixed_text(400_000, 901),   # larger first ...
        workloads.hard_case_text(100_000, 902),    # ... then hard cases: more pending fields
                                                   # than the fixed queue holds
        workloads.uniform_text(1000, 903),         # ... then a much smaller one
    ]
    for text in inputs:
        t = _device_text(text)
        rb, rs = oracle.parse_buffer(text)
        ref = _run(lib.fp_parse_f64, t)
        got = _run(lib.fp_parse_f64_noalloc, t)
        assert got[0] == rb.size and ref[0] == rb.size and rb.size > 0
        assert np.array_equal(got[1], rb) and np.array_equal(got[2], rs)
        assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    # and once more with the first input, after the others left their state
    rb, rs = oracle.parse_buffer(inputs[0])
    got = _run(lib.fp_parse_f64_noalloc, _device_text(inputs[0]))
    assert np.array_equal(got[1], rb) and np.array_equal(got[2], rs)


def test_noalloc_overflows_its_fixed_queue_into_the_chunk_scan():
    # hard cases send most fields to the fallback kernel: more than the fixed
    # array's queue entries, so the rest are found by scanning their chunks
    text = workloads.hard_case_text(100_000, 904)
    t = _device_text(text)
    s_before = fp.stats(reset=True)
    ref = _run(_lib.load().fp_parse_f64, t)
    pending = fp.stats(reset=True)["fallback"]
    assert pending > NOALLOC_QUEUE, (pending, s_before)
    rb, rs = oracle.parse_buffer(text)
    got = _run(_lib.load().fp_parse_f64_noalloc, t)
    assert got[0] == rb.size == ref[0]
    assert np.array_equal(got[1], rb) and np.array_equal(got[2], rs)


def test_noalloc_allocates_nothing_once_set_up():
    lib = _lib.load()
    text = workloads.hard_case_text(20_000, 905) + b"\n" + workloads.bulk_mixed_text(50_000, 906)
    t = _device_text(text)
    outs = [_outputs(t.numel(), t.device) for _ in range(2)]
    assert _call(lib.fp_parse_f64_noalloc, t, outs[0]) == _lib.FP_OK  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    stats0 = torch.cuda.memory_stats()
    for o in outs:  # two calls in a row
        assert _call(lib.fp_parse_f64_noalloc, t, o) == _lib.FP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    stats1 = torch.cuda.memory_stats()
    assert free1 == free0
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key) == stats0.get(key), key
    rb, rs = oracle.parse_buffer(text)
    for out, st, cnt in outs:
        assert int(cnt.item()) == rb.size
        assert np.array_equal(out[:rb.size].cpu().numpy().view(np.uint64), rb)
        assert np.array_equal(st[:rb.size].cpu().numpy(), rs)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    lib = _lib.load()
    chunk = fp.get_config()["chunk_bytes"]
    # a text one byte longer than the array's chunks cover ("1\n" repeated),
    # with real buffers of that size behind every pointer: nothing would be
    # out of bounds even if the check were missing
    too_long = NOALLOC_MAX_CHUNKS * chunk + 1
    t = torch.tensor([ord("1"), ord("\n")], dtype=torch.uint8,
                     device="cuda").repeat(too_long // 2 + 1)[:too_long]
    assert t.data_ptr() % 16 == 0
    outs = _outputs(too_long, t.device)
    assert _call(lib.fp_parse_f64_noalloc, t, outs) == _lib.FP_ERR_CAPACITY
    torch.cuda.synchronize()
    assert int(outs[2].item()) == 0 and float(outs[0][0].item()) == -7.0  # nothing ran
    # one byte shorter fits: 2^k fields "1"
    short = t[:too_long - 1]
    assert _call(lib.fp_parse_f64_noalloc, short, outs) == _lib.FP_OK
    torch.cuda.synchronize()
    n = (too_long - 1) // 2
    out, st, cnt = outs
    assert int(cnt.item()) == n
    assert bool((out[:n] == 1.0).all()) and bool((st[:n] == 0).all())
    del t, outs, short, out, st, cnt
    torch.cuda.empty_cache()
