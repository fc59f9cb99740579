"""Calls of every kind queued back to back on one stream, with no
synchronisation between them.  Each call's parse kernel is a programmatic
dependent launch that the kernel before it (the previous call's fallback
kernel) releases as it starts: it is set up while that call still runs and
waits on the device before it reads or writes anything, including the
stream's control block, which the previous fallback kernel resets as it
ends.  The calls mix the decimal, binary32, hexadecimal, JSON and
column-major kernels, a hard-case text whose fallback kernel has most of
the work, a small text (4 KiB chunks, a one-block-per-SM fallback launch)
and the allocation-free entry point (its own fixed scratch).  Every output
must equal the oracle's, bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import paper_2101_11408_gb300 as fp
from paper_2101_11408_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu


def _dev(text: bytes) -> torch.Tensor:
    return torch.frombuffer(bytearray(text), dtype=torch.uint8).cuda()


def _outs(n: int, f32: bool = False):
    n = max(n, 1)
    return (torch.full((n,), -7.0, dtype=torch.float32 if f32 else torch.float64, device="cuda"),
            torch.full((n,), 0xEE, dtype=torch.uint8, device="cuda"),
            torch.zeros(1, dtype=torch.int64, device="cuda"))


def test_calls_of_every_kind_back_to_back_on_one_stream():
    bulk = workloads.bulk_mixed_text(200000, workloads.SEED_BASE + 120)
    hexs = workloads.hex_float_text(100000, workloads.SEED_BASE + 121)
    hard = workloads.hard_case_text(20000, workloads.SEED_BASE + 122)
    small = workloads.uniform_text(3000, workloads.SEED_BASE + 123)
    K = 4
    lines = workloads.uniform_lines(40000, workloads.SEED_BASE + 124)
    csv = "\n".join(",".join(lines[r * K:(r + 1) * K]) for r in range(len(lines) // K)).encode()
    rows_cap = len(lines) // K + 1
    texts = {"bulk": _dev(bulk), "hex": _dev(hexs), "hard": _dev(hard), "small": _dev(small),
             "csv": _dev(csv)}
    # (kind, text name, outputs), in queue order: two rounds, the second in
    # another order, so each kind follows several others
    order = ["bulk", "hex", "hard", "f32", "json", "columns", "small", "noalloc", "hard",
             "columns", "f32", "small", "hex", "noalloc", "json", "bulk", "hard"]
    src = {"bulk": "bulk", "hex": "hex", "hard": "hard", "f32": "bulk", "json": "bulk",
           "columns": "csv", "small": "small", "noalloc": "bulk"}
    jobs = []
    for kind in order:
        t = texts[src[kind]]
        n = K * rows_cap if kind == "columns" else t.numel()
        jobs.append((kind, _outs(n, f32=(kind == "f32"))))
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    lib = _lib.load()
    for kind, (out, st, cnt) in jobs:
        t = texts[src[kind]]
        if kind in ("bulk", "hard", "small"):
            fp.parse_f64_into(t, out, st, cnt, stream=s)
        elif kind == "f32":
            fp.parse_f32_into(t, out, st, cnt, stream=s)
        elif kind == "hex":
            fp.parse_ex_into(t, out, st, cnt, grammar="hex", stream=s)
        elif kind == "json":
            fp.parse_ex_into(t, out, st, cnt, grammar="json", stream=s)
        elif kind == "columns":
            fp.parse_ex_into(t, out, st, cnt, delim=b",", columns=K, rows_cap=rows_cap, stream=s)
        else:
            rc = lib.fp_parse_f64_noalloc(t.data_ptr(), t.numel(), b"\n", out.data_ptr(),
                                          st.data_ptr(), cnt.data_ptr(), s.cuda_stream)
            assert rc == _lib.FP_OK, _lib.strerror(rc)
    s.synchronize()
    assert fp.get_error(stream=s) == 0
    want = {}
    for kind, (out, st, cnt) in jobs:
        text = {"bulk": bulk, "hex": hexs, "hard": hard, "small": small, "csv": csv}[src[kind]]
        if kind not in want:
            if kind == "columns":
                rb, rs = oracle.parse_buffer(csv, b",")
                want[kind] = (rb.size,) + oracle.columnar(csv, rb, rs, K, rows_cap, b",")
            else:
                grammar = {"hex": oracle.GRAMMAR_HEX, "json": oracle.GRAMMAR_JSON}.get(
                    kind, oracle.GRAMMAR_DEFAULT)
                rb, rs = oracle.parse_buffer(text, f32=(kind == "f32"), grammar=grammar)
                want[kind] = (rb.size, rb, rs)
        n_want, wb, ws = want[kind]
        assert int(cnt.item()) == n_want, kind
        if kind == "columns":
            got = out.cpu().numpy().view(np.uint64)
            gst = st.cpu().numpy()
            filled = ws != 0xEE
            assert np.array_equal(gst, ws) and np.array_equal(got[filled], wb[filled]), kind
        else:
            got = out[:n_want].cpu().numpy().view(np.uint32 if kind == "f32" else np.uint64)
            assert np.array_equal(got, wb) and np.array_equal(st[:n_want].cpu().numpy(), ws), kind
