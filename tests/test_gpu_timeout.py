"""A bounded device wait that runs out, on purpose and without a fault.

Every wait in the parse kernel (the decoupled look-back's wait for an earlier
chunk's word, the wait for a staged tile) gives up after a time limit,
records FP_ERR_TIMEOUT in the stream's error word and lets the kernel
finish.  The test hook fp_test_arm_stalled_lookback makes the next call skip
chunk 0, so the look-back of the chunks after it waits for a word that
nothing writes; with a limit of a few milliseconds the call must end, report
FP_ERR_TIMEOUT through fp_get_error, and leave the stream usable: the next
call is bit-exact against the oracle again and reports no error.
"""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def _parse_checked(t, text, stream):
    vals, st = fp.parse_f64(t, stream=stream)
    torch.cuda.synchronize()
    rb, rs = oracle.parse_buffer(text)
    assert np.array_equal(vals.cpu().numpy().view(np.uint64), rb)
    assert np.array_equal(st.cpu().numpy(), rs)


@pytest.mark.parametrize("limit_ms", [2, 20])
def test_stalled_lookback_times_out_and_the_next_call_recovers(limit_ms):
    lib = _lib.load()
    text = workloads.uniform_text(60_000, 931)  # about 1.1 MB: hundreds of 4 KiB chunks
    t = torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _parse_checked(t, text, stream)
        assert fp.get_error(stream) == _lib.FP_OK
        rc = lib.fp_test_arm_stalled_lookback(stream.cuda_stream, limit_ms * 1_000_000)
        assert rc == _lib.FP_OK
        out = torch.empty(t.numel(), dtype=torch.float64, device=t.device)
        st = torch.empty(t.numel(), dtype=torch.uint8, device=t.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=t.device)
        t0 = time.perf_counter()
        fp.parse_f64_into(t, out, st, cnt, stream=stream)
        stream.synchronize()
        elapsed = time.perf_counter() - t0
        # the waits gave up after the short limit, not the 2 s default
        assert elapsed < 1.5, elapsed
        assert fp.get_error(stream) == _lib.FP_ERR_TIMEOUT
        assert fp.get_error(stream) == _lib.FP_OK  # read once, then cleared
        # the stream and its scratch are usable again
        _parse_checked(t, text, stream)
        assert fp.get_error(stream) == _lib.FP_OK


def test_the_hook_rejects_limits_beyond_the_default():
    lib = _lib.load()
    s = torch.cuda.current_stream().cuda_stream
    assert lib.fp_test_arm_stalled_lookback(s, 0) == _lib.FP_ERR_ARG
    assert lib.fp_test_arm_stalled_lookback(s, 2_000_000_001) == _lib.FP_ERR_ARG
