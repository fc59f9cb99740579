"""GB300-native bulk parser: ASCII decimal text -> nearest binary64, bit-exact.

Python front end of libfpparse.so (C ABI in include/fpparse.h).  PyTorch
supplies device memory and streams; every step of the parse runs in the
library's sm_103a kernels.  If the library cannot be loaded these functions
raise: there is no CPU implementation behind them.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import (STATUS_INVALID, STATUS_OK, STATUS_OVERFLOW, STATUS_UNDERFLOW, Config,
                   FpError, Stats)

__all__ = ["BatchPlan", "Server", "parse_ex", "parse_ex_into", "parse_f32", "parse_f32_into",
           "parse_f64", "parse_f64_into", "parse_f64_host", "parse_f64_host_into", "parse_f64_batch",
           "parse_f64_batch_into", "max_fields", "stats", "get_error", "set_config",
           "get_config", "autotune", "timing_enable", "timing_read", "shutdown", "library_path", "FpError", "STATUS_OK",
           "STATUS_INVALID", "STATUS_OVERFLOW", "STATUS_UNDERFLOW"]


def library_path() -> str:
    return _lib.library_path()


def _delim_byte(delim) -> bytes:
    if isinstance(delim, str):
        delim = delim.encode()
    if not isinstance(delim, (bytes, bytearray)) or len(delim) != 1:
        raise ValueError("delim must be one byte")
    return bytes(delim)


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _check_text(text: torch.Tensor) -> None:
    if not isinstance(text, torch.Tensor) or text.dtype != torch.uint8 or text.dim() != 1:
        raise TypeError("text must be a 1-D torch.uint8 tensor")
    if not text.is_cuda:
        raise TypeError("text must be a CUDA tensor (use parse_f64_host for host data)")
    if not text.is_contiguous():
        raise TypeError("text must be contiguous")


# dtypes of a field-count tensor (8-byte integers)
_COUNT_DTYPES = (torch.int64,) + ((torch.uint64,) if hasattr(torch, "uint64") else ())
# host arrays: the torch and numpy forms of each element type
_HOST_TYPES = {"uint8": (torch.uint8, np.dtype(np.uint8)),
               "float64": (torch.float64, np.dtype(np.float64))}


def _check_out(t, dtypes, need: int, dev: int, name: str) -> None:
    """An array the library writes: a contiguous tensor of one of `dtypes` on
    CUDA device `dev` with at least `need` entries (the kernels write through
    its address, so a tensor elsewhere or too small is refused before the
    call).  Cheap on the accepted path: it runs on every call."""
    if not isinstance(t, torch.Tensor) or t.dtype not in dtypes:
        raise TypeError("%s must be a tensor of dtype %s"
                        % (name, " or ".join(str(d) for d in dtypes)))
    if not t.is_cuda or t.get_device() != dev:
        raise TypeError("%s must be on cuda:%d, not %s" % (name, dev, t.device))
    if not t.is_contiguous():
        raise TypeError("%s must be contiguous" % name)
    if t.numel() < need:
        raise ValueError("%s needs at least %d entries, has %d" % (name, need, t.numel()))


def _host_array(a, kind: str, need: int, name: str, writable: bool = True) -> int:
    """Address of a host array (numpy array or CPU tensor) of element type
    `kind` ("uint8" or "float64"), contiguous, with at least `need` entries."""
    tdt, ndt = _HOST_TYPES[kind]
    if isinstance(a, torch.Tensor):
        if not a.is_cpu or a.dtype is not tdt:
            raise TypeError("%s must be a CPU tensor of %s" % (name, kind))
        if not a.is_contiguous():
            raise TypeError("%s must be contiguous" % name)
        size, addr = a.numel(), a.data_ptr()
    elif isinstance(a, np.ndarray):
        if a.dtype != ndt or not a.flags.c_contiguous:
            raise TypeError("%s must be a contiguous numpy array of %s" % (name, kind))
        if writable and not a.flags.writeable:
            raise TypeError("%s must be writable" % name)
        size, addr = a.size, a.ctypes.data
    else:
        raise TypeError("%s must be a numpy array or a CPU tensor" % name)
    if size < need:
        raise ValueError("%s needs at least %d entries, has %d" % (name, need, size))
    return addr


def max_fields(nbytes: int) -> int:
    return int(_lib.load().fp_max_fields(nbytes))


def parse_f64_into(text: torch.Tensor, out_f64: torch.Tensor, out_status: torch.Tensor,
                   out_count: torch.Tensor, delim=b"\n", stream=None) -> None:
    """Queue the parse of `text` on `stream` (asynchronous).

    out_f64 (float64), out_status (uint8) need max_fields(len) entries on the
    same device; out_count is a one-element int64/uint64 device tensor.
    """
    _check_text(text)
    n, dev = text.numel(), text.get_device()
    _check_out(out_f64, (torch.float64,), n, dev, "out_f64")
    _check_out(out_status, (torch.uint8,), n, dev, "out_status")
    _check_out(out_count, _COUNT_DTYPES, 1, dev, "out_count")
    lib = _lib.load()
    rc = lib.fp_parse_f64(text.data_ptr() if n else None, n, _delim_byte(delim),
                          out_f64.data_ptr() if n else None,
                          out_status.data_ptr() if n else None, out_count.data_ptr(),
                          _stream_handle(stream))
    _lib.check(rc, "fp_parse_f64")


def parse_f64(text: torch.Tensor, delim=b"\n", stream=None):
    """Parse every field of a device buffer.  Returns (values float64,
    status uint8) device tensors of the field count (synchronises)."""
    _check_text(text)
    dev = text.device
    cap = max(text.numel(), 1)
    out = torch.empty(cap, dtype=torch.float64, device=dev)
    st = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    parse_f64_into(text, out, st, cnt, delim, stream)
    n = int(cnt.item()) if stream is None else None
    if n is None:
        stream.synchronize()
        n = int(cnt.item())
    return out[:n], st[:n]


def parse_f32_into(text: torch.Tensor, out_f32: torch.Tensor, out_status: torch.Tensor,
                   out_count: torch.Tensor, delim=b"\n", stream=None) -> None:
    """As parse_f64_into, to binary32 (out_f32 float32)."""
    _check_text(text)
    n, dev = text.numel(), text.get_device()
    _check_out(out_f32, (torch.float32,), n, dev, "out_f32")
    _check_out(out_status, (torch.uint8,), n, dev, "out_status")
    _check_out(out_count, _COUNT_DTYPES, 1, dev, "out_count")
    lib = _lib.load()
    rc = lib.fp_parse_f32(text.data_ptr() if n else None, n, _delim_byte(delim),
                          out_f32.data_ptr() if n else None,
                          out_status.data_ptr() if n else None, out_count.data_ptr(),
                          _stream_handle(stream))
    _lib.check(rc, "fp_parse_f32")


def parse_f32(text: torch.Tensor, delim=b"\n", stream=None):
    """Parse every field of a device buffer to binary32.  Returns (values
    float32, status uint8) device tensors of the field count (synchronises)."""
    _check_text(text)
    dev = text.device
    cap = max(text.numel(), 1)
    out = torch.empty(cap, dtype=torch.float32, device=dev)
    st = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    parse_f32_into(text, out, st, cnt, delim, stream)
    if stream is not None:
        stream.synchronize()
    n = int(cnt.item())
    return out[:n], st[:n]


_GRAMMARS = {"decimal": 0, "hex": 1, "json": 2}


def parse_ex_into(text: torch.Tensor, out_values: torch.Tensor, out_status: torch.Tensor,
                  out_count: torch.Tensor, delim=b"\n", grammar: str = "decimal",
                  columns: int = 0, rows_cap: int = 0, stream=None) -> None:
    """fp_parse_ex: out_values float64 or float32 picks the format; grammar
    'decimal', 'hex' or 'json'; columns K >= 2 stores field i at
    (i mod K) * rows_cap + i div K."""
    _check_text(text)
    n = text.numel()
    need = columns * rows_cap if columns else n
    dev = text.get_device()
    _check_out(out_values, (torch.float64, torch.float32), need, dev, "out_values")
    _check_out(out_status, (torch.uint8,), need, dev, "out_status")
    _check_out(out_count, _COUNT_DTYPES, 1, dev, "out_count")
    opt = _lib.Options(_delim_byte(delim), 1 if out_values.dtype == torch.float32 else 0,
                       _GRAMMARS[grammar], 0, columns, rows_cap)
    rc = _lib.load().fp_parse_ex(text.data_ptr() if n else None, n, ctypes.byref(opt),
                                 out_values.data_ptr() if need else None,
                                 out_status.data_ptr() if need else None, out_count.data_ptr(),
                                 _stream_handle(stream))
    _lib.check(rc, "fp_parse_ex")


def parse_ex(text: torch.Tensor, delim=b"\n", f32: bool = False, grammar: str = "decimal",
             columns: int = 0, rows_cap: int = 0, stream=None):
    """fp_parse_ex on a device buffer.  Field order: (values, status) of the
    field count; column-major: (values, status) of shape (columns, rows_cap)
    (entries no field reaches are left as allocated).  Synchronises."""
    _check_text(text)
    dev = text.device
    cap = columns * rows_cap if columns else max(text.numel(), 1)
    out = torch.empty(cap, dtype=torch.float32 if f32 else torch.float64, device=dev)
    st = torch.full((cap,), 0xEE, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    parse_ex_into(text, out, st, cnt, delim, grammar, columns, rows_cap, stream)
    if stream is not None:
        stream.synchronize()
    n = int(cnt.item())
    if columns:
        return out.view(columns, rows_cap), st.view(columns, rows_cap), n
    return out[:n], st[:n]


def parse_f64_host_into(host_text, host_f64, host_status, delim=b"\n", stream=None) -> int:
    """End-to-end parse of host memory through the C ABI (fp_parse_f64_host):
    host_text is a uint8 numpy array or CPU tensor (pinned copies fastest),
    host_f64 / host_status receive the results.  Returns the field count."""
    n = host_text.numel() if isinstance(host_text, torch.Tensor) else getattr(host_text, "size", 0)
    p_text = _host_array(host_text, "uint8", n, "host_text", writable=False)
    p_f64 = _host_array(host_f64, "float64", n, "host_f64")  # max_fields(n) entries
    p_st = _host_array(host_status, "uint8", n, "host_status")
    cnt = ctypes.c_uint64()
    rc = _lib.load().fp_parse_f64_host(p_text if n else None, n, _delim_byte(delim),
                                       p_f64 if n else None, p_st if n else None,
                                       ctypes.byref(cnt), _stream_handle(stream))
    _lib.check(rc, "fp_parse_f64_host")
    return int(cnt.value)


def parse_f64_host(data, delim=b"\n", stream=None):
    """Parse host bytes end to end.  Returns numpy (values, status)."""
    if isinstance(data, (bytes, bytearray, memoryview)):
        arr = np.frombuffer(bytearray(data), dtype=np.uint8)
    else:
        arr = np.ascontiguousarray(data, dtype=np.uint8)
    cap = max(arr.size, 1)
    vals = np.empty(cap, dtype=np.float64)
    st = np.empty(cap, dtype=np.uint8)
    n = parse_f64_host_into(arr, vals, st, delim, stream)
    return vals[:n], st[:n]


def _batch_args(texts, out_f64, out_status, out_offsets, out_counts):
    """Checked ctypes arrays (text pointers, lengths, output offsets) of a
    batch: device buffers on one device, outputs there with room for
    out_offsets[-1] entries, one count per buffer."""
    nbuf = len(texts)
    if nbuf == 0:
        raise ValueError("no buffers")
    for t in texts:
        _check_text(t)
        if t.get_device() != texts[0].get_device():
            raise TypeError("all buffers must be on one device")
    offsets = [int(o) for o in out_offsets]
    if len(offsets) != nbuf + 1:
        raise ValueError("out_offsets needs nbuf + 1 entries")
    dev = texts[0].get_device()
    _check_out(out_f64, (torch.float64,), offsets[-1], dev, "out_f64")
    _check_out(out_status, (torch.uint8,), offsets[-1], dev, "out_status")
    _check_out(out_counts, _COUNT_DTYPES, nbuf, dev, "out_counts")
    ptrs = (ctypes.c_void_p * nbuf)(*[t.data_ptr() if t.numel() else None for t in texts])
    lens = (ctypes.c_size_t * nbuf)(*[t.numel() for t in texts])
    offs = (ctypes.c_uint64 * (nbuf + 1))(*offsets)
    return ptrs, lens, offs


def parse_f64_batch_into(texts, out_f64: torch.Tensor, out_status: torch.Tensor,
                         out_offsets, out_counts: torch.Tensor, delim=b"\n",
                         stream=None) -> None:
    """Queue one persistent launch over many device buffers.

    out_offsets: nbuf+1 host integers; buffer b owns output entries
    [out_offsets[b], out_offsets[b+1]).  out_counts: nbuf-element device
    tensor receiving the field counts.
    """
    ptrs, lens, offs = _batch_args(texts, out_f64, out_status, out_offsets, out_counts)
    nbuf = len(texts)
    lib = _lib.load()
    rc = lib.fp_parse_f64_batch(ptrs, lens, nbuf, _delim_byte(delim), out_f64.data_ptr(),
                                out_status.data_ptr(), offs, out_counts.data_ptr(),
                                _stream_handle(stream))
    _lib.check(rc, "fp_parse_f64_batch")


def parse_f64_batch(texts, delim=b"\n", stream=None):
    """Parse many device buffers in one launch.  Returns a list of
    (values, status) device tensors, one per buffer (synchronises)."""
    offs = [0]
    for t in texts:
        offs.append(offs[-1] + max(t.numel(), 0))
    dev = texts[0].device
    cap = max(offs[-1], 1)
    out = torch.empty(cap, dtype=torch.float64, device=dev)
    st = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(len(texts), dtype=torch.int64, device=dev)
    parse_f64_batch_into(texts, out, st, offs, cnt, delim, stream)
    if stream is not None:
        stream.synchronize()
    counts = cnt.cpu().tolist()
    return [(out[offs[b]:offs[b] + counts[b]], st[offs[b]:offs[b] + counts[b]])
            for b in range(len(texts))]


class BatchPlan:
    """A fixed set of device buffers parsed by one replayable launch
    (fp_batch_plan_*); with graph=True the launch is one CUDA graph replay.
    Keeps references to the buffers and outputs."""

    def __init__(self, texts, out_f64, out_status, out_offsets, out_counts, delim=b"\n",
                 graph=False):
        ptrs, lens, offs = _batch_args(texts, out_f64, out_status, out_offsets, out_counts)
        nbuf = len(texts)
        self._keep = (texts, out_f64, out_status, out_counts)
        self.capacity = offs[nbuf] - offs[0]  # the packed results fit in this many entries
        self._h = ctypes.c_void_p()
        _lib.check(_lib.load().fp_batch_plan_create(ptrs, lens, nbuf, _delim_byte(delim),
                                                    out_f64.data_ptr(), out_status.data_ptr(),
                                                    offs, out_counts.data_ptr(),
                                                    1 if graph else 0, ctypes.byref(self._h)),
                   "fp_batch_plan_create")

    def launch(self, stream=None) -> None:
        _lib.check(_lib.load().fp_batch_plan_launch(self._h, _stream_handle(stream)),
                   "fp_batch_plan_launch")

    def gather(self, dst_f64: torch.Tensor, dst_status: torch.Tensor, dst_total: torch.Tensor,
               stream=None) -> None:
        """Pack the last launch's results in buffer order into dst_f64 /
        dst_status (float64 / uint8 device tensors with room for the total,
        at most self.capacity entries) and their number into dst_total (one
        int64 device element), on the stream, without synchronising
        (fp_batch_plan_gather)."""
        dev = self._keep[0][0].get_device()
        # room for the total: the caller may know it (fixed inputs); it is at
        # most the plan's output capacity, self.capacity
        _check_out(dst_f64, (torch.float64,), 0, dev, "dst_f64")
        _check_out(dst_status, (torch.uint8,), 0, dev, "dst_status")
        _check_out(dst_total, _COUNT_DTYPES, 1, dev, "dst_total")
        _lib.check(_lib.load().fp_batch_plan_gather(self._h, dst_f64.data_ptr(),
                                                    dst_status.data_ptr(), dst_total.data_ptr(),
                                                    _stream_handle(stream)),
                   "fp_batch_plan_gather")

    def close(self) -> None:
        if self._h:
            _lib.load().fp_batch_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server on the current device
    (fp_server_*).  Requests are host tensors: uint8 text, float64 values and
    uint8 statuses (pinned memory copies fastest); the first min(fields,
    len(values), len(statuses)) results are written.  The server keeps
    references to the tensors until they are waited for."""

    def __init__(self, device_budget: int = 40_000_000_000, max_batch: int = 1024,
                 max_inflight: int = 4, delim=b"\n", launch_bytes: int = 0):
        cfg = _lib.ServerConfig(device_budget, max_batch, max_inflight, _delim_byte(delim),
                                launch_bytes)
        self._h = ctypes.c_void_p()
        _lib.check(_lib.load().fp_server_create(ctypes.byref(cfg), ctypes.byref(self._h)),
                   "fp_server_create")
        self._keep = {}

    def submit(self, host_text: torch.Tensor, host_f64: torch.Tensor,
               host_status: torch.Tensor) -> int:
        for t, dt in ((host_text, torch.uint8), (host_f64, torch.float64),
                      (host_status, torch.uint8)):
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous():
                raise ValueError("server requests are contiguous host tensors")
        n = host_text.numel()
        cap = min(host_f64.numel(), host_status.numel())
        rid = ctypes.c_uint64()
        _lib.check(_lib.load().fp_server_submit(self._h, host_text.data_ptr() if n else None, n,
                                                host_f64.data_ptr() if cap else None,
                                                host_status.data_ptr() if cap else None, cap,
                                                ctypes.byref(rid)), "fp_server_submit")
        self._keep[rid.value] = (host_text, host_f64, host_status)
        return rid.value

    def wait(self, request_id: int, timeout_s: float | None = None) -> dict | None:
        """Info dict of a finished request (count, error, batch_size and the
        CLOCK_MONOTONIC ns of submit/admit/launch/done), or None on timeout."""
        info = _lib.RequestInfo()
        t = -1 if timeout_s is None else int(timeout_s * 1e9)
        rc = _lib.load().fp_server_wait(self._h, request_id, t, ctypes.byref(info))
        if rc == _lib.FP_ERR_TIMEOUT:
            return None
        self._keep.pop(request_id, None)
        if rc != _lib.FP_OK and info.error == 0:
            _lib.check(rc, "fp_server_wait")
        return info.as_dict()

    def stats(self) -> dict:
        s = _lib.ServerStats()
        _lib.check(_lib.load().fp_server_get_stats(self._h, ctypes.byref(s)), "fp_server_get_stats")
        return s.as_dict()

    def close(self) -> None:
        if self._h:
            _lib.load().fp_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats(reset: bool = False, stream=None) -> dict:
    s = Stats()
    _lib.check(_lib.load().fp_get_stats(ctypes.byref(s), int(reset), _stream_handle(stream)),
               "fp_get_stats")
    return s.as_dict()


def get_error(stream=None) -> int:
    return int(_lib.load().fp_get_error(_stream_handle(stream)))


def set_config(chunk_bytes=None, ctas_per_sm=None, fallback_queue=None) -> dict:
    cur = get_config()
    c = Config(chunk_bytes if chunk_bytes is not None else cur["chunk_bytes"],
               ctas_per_sm if ctas_per_sm is not None else cur["ctas_per_sm"],
               fallback_queue if fallback_queue is not None else cur["fallback_queue"])
    _lib.check(_lib.load().fp_set_config(ctypes.byref(c)), "fp_set_config")
    return get_config()


def get_config() -> dict:
    c = Config()
    _lib.check(_lib.load().fp_get_config(ctypes.byref(c)), "fp_get_config")
    return {"chunk_bytes": c.chunk_bytes, "ctas_per_sm": c.ctas_per_sm,
            "fallback_queue": c.fallback_queue}


def autotune(text: torch.Tensor, delim=b"\n", cache_path: str | None = None) -> dict:
    _check_text(text)
    c = Config()
    _lib.check(_lib.load().fp_autotune(text.data_ptr(), text.numel(), _delim_byte(delim),
                                       cache_path.encode() if cache_path else None,
                                       ctypes.byref(c)), "fp_autotune")
    return {"chunk_bytes": c.chunk_bytes, "ctas_per_sm": c.ctas_per_sm,
            "fallback_queue": c.fallback_queue}


def timing_enable(on: bool = True, every: int = 1) -> None:
    """Record CUDA events around each kernel of every `every`-th later call on
    a stream (see timing_read); on=False turns it off."""
    if on and every < 1:
        raise ValueError("every must be at least 1")
    _lib.check(_lib.load().fp_timing_enable(int(every) if on else 0), "fp_timing_enable")


def timing_read(stream=None) -> dict:
    """Summed device time of the kernels of the timed calls on `stream` since
    the last read: {"parse_ms", "fallback_ms", "calls"} (waits for them)."""
    a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint64()
    _lib.check(_lib.load().fp_timing_read(_stream_handle(stream), ctypes.byref(a),
                                          ctypes.byref(b), ctypes.byref(n)), "fp_timing_read")
    return {"parse_ms": a.value, "fallback_ms": b.value, "calls": int(n.value)}


def shutdown() -> None:
    _lib.check(_lib.load().fp_shutdown(), "fp_shutdown")
