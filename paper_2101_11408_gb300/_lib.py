"""ctypes binding of libfpparse.so (include/fpparse.h).  Argument marshalling
only: every step of the parse runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

FP_OK, FP_ERR_ARG, FP_ERR_CAPACITY, FP_ERR_CUDA, FP_ERR_BUDGET, FP_ERR_TIMEOUT, \
    FP_ERR_INTERNAL = range(7)
STATUS_OK, STATUS_INVALID, STATUS_OVERFLOW, STATUS_UNDERFLOW, STATUS_BAD_SHAPE = range(5)
FORMAT_F64, FORMAT_F32 = 0, 1
GRAMMAR_DECIMAL, GRAMMAR_HEX, GRAMMAR_JSON = 0, 1, 2

# every symbol include/*.h declares (fpparse_test.h: test hooks; fpparse_bench.h:
# trace replay for measurements)
EXPORTS = ["fp_max_fields", "fp_parse_f64", "fp_parse_f32", "fp_parse_ex", "fp_parse_f64_batch", "fp_get_stats",
           "fp_get_error", "fp_set_config", "fp_get_config", "fp_autotune", "fp_timing_enable",
           "fp_timing_read", "fp_parse_f64_host", "fp_parse_f64_noalloc", "fp_batch_plan_create",
           "fp_batch_plan_launch", "fp_batch_plan_destroy", "fp_batch_plan_gather",
           "fp_server_create", "fp_server_submit",
           "fp_server_wait", "fp_server_get_stats", "fp_server_destroy", "fp_shutdown",
           "fp_strerror", "fp_test_arm_stalled_lookback", "fp_replay_server", "fp_replay_plain"]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "calls", "fields", "bytes", "one_multiply", "two_multiplies", "long_fields",
        "long_settled", "fallback", "fallback_bignum", "queue_overflow", "general_tokenizer")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Config(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("fallback_queue", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("delim", ctypes.c_char),
                ("launch_bytes", ctypes.c_uint64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("error", ctypes.c_int32),
                ("batch_size", ctypes.c_uint32), ("submit_ns", ctypes.c_int64),
                ("admit_ns", ctypes.c_int64), ("launch_ns", ctypes.c_int64),
                ("done_ns", ctypes.c_int64)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "submitted", "completed", "launches", "bytes", "fields", "peak_units", "peak_requests",
        "max_batch_seen")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class Options(ctypes.Structure):
    _fields_ = [("delim", ctypes.c_char), ("format", ctypes.c_uint8), ("grammar", ctypes.c_uint8),
                ("reserved", ctypes.c_uint8), ("columns", ctypes.c_uint32),
                ("rows_cap", ctypes.c_uint64)]


class ReplayBody(ctypes.Structure):
    _fields_ = [("host_text", ctypes.c_void_p), ("len", ctypes.c_size_t),
                ("host_f64", ctypes.c_void_p), ("host_status", ctypes.c_void_p),
                ("out_cap", ctypes.c_size_t)]


class FpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (code %d)" % (where, strerror(code), code))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it in-tree if absent).  Raises if it
    cannot be loaded: there is no fallback implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError("libfpparse.so is not built (%s)" % path)
            _build.build_library()
        lib = ctypes.CDLL(path)
        vp, sz, u8p = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p
        lib.fp_max_fields.argtypes = [sz]
        lib.fp_max_fields.restype = sz
        lib.fp_parse_f64.argtypes = [vp, sz, ctypes.c_char, vp, u8p, vp, vp]
        lib.fp_parse_f64.restype = ctypes.c_int
        lib.fp_parse_f32.argtypes = [vp, sz, ctypes.c_char, vp, u8p, vp, vp]
        lib.fp_parse_f32.restype = ctypes.c_int
        lib.fp_parse_ex.argtypes = [vp, sz, ctypes.POINTER(Options), vp, u8p, vp, vp]
        lib.fp_parse_ex.restype = ctypes.c_int
        lib.fp_parse_f64_batch.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_char, vp, u8p,
                                           vp, vp, vp]
        lib.fp_parse_f64_batch.restype = ctypes.c_int
        lib.fp_get_stats.argtypes = [ctypes.POINTER(Stats), ctypes.c_int, vp]
        lib.fp_get_stats.restype = ctypes.c_int
        lib.fp_get_error.argtypes = [vp]
        lib.fp_get_error.restype = ctypes.c_int
        lib.fp_set_config.argtypes = [ctypes.POINTER(Config)]
        lib.fp_set_config.restype = ctypes.c_int
        lib.fp_get_config.argtypes = [ctypes.POINTER(Config)]
        lib.fp_get_config.restype = ctypes.c_int
        lib.fp_autotune.argtypes = [vp, sz, ctypes.c_char, ctypes.c_char_p,
                                    ctypes.POINTER(Config)]
        lib.fp_autotune.restype = ctypes.c_int
        lib.fp_timing_enable.argtypes = [ctypes.c_int]
        lib.fp_timing_enable.restype = ctypes.c_int
        lib.fp_timing_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_uint64)]
        lib.fp_timing_read.restype = ctypes.c_int
        lib.fp_parse_f64_host.argtypes = [vp, sz, ctypes.c_char, vp, u8p, vp, vp]
        lib.fp_parse_f64_host.restype = ctypes.c_int
        lib.fp_parse_f64_noalloc.argtypes = [vp, sz, ctypes.c_char, vp, u8p, vp, vp]
        lib.fp_parse_f64_noalloc.restype = ctypes.c_int
        lib.fp_batch_plan_create.argtypes = [vp, vp, ctypes.c_uint32, ctypes.c_char, vp, u8p,
                                             vp, vp, ctypes.c_uint32,
                                             ctypes.POINTER(ctypes.c_void_p)]
        lib.fp_batch_plan_create.restype = ctypes.c_int
        lib.fp_batch_plan_launch.argtypes = [vp, vp]
        lib.fp_batch_plan_launch.restype = ctypes.c_int
        lib.fp_batch_plan_destroy.argtypes = [vp]
        lib.fp_batch_plan_destroy.restype = ctypes.c_int
        lib.fp_batch_plan_gather.argtypes = [vp, vp, u8p, vp, vp]
        lib.fp_batch_plan_gather.restype = ctypes.c_int
        lib.fp_server_create.argtypes = [ctypes.POINTER(ServerConfig),
                                         ctypes.POINTER(ctypes.c_void_p)]
        lib.fp_server_create.restype = ctypes.c_int
        lib.fp_server_submit.argtypes = [vp, vp, sz, vp, u8p, sz,
                                         ctypes.POINTER(ctypes.c_uint64)]
        lib.fp_server_submit.restype = ctypes.c_int
        lib.fp_server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64,
                                       ctypes.POINTER(RequestInfo)]
        lib.fp_server_wait.restype = ctypes.c_int
        lib.fp_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        lib.fp_server_get_stats.restype = ctypes.c_int
        lib.fp_server_destroy.argtypes = [vp]
        lib.fp_server_destroy.restype = ctypes.c_int
        lib.fp_shutdown.argtypes = []
        lib.fp_shutdown.restype = ctypes.c_int
        lib.fp_replay_server.argtypes = [vp, ctypes.POINTER(ReplayBody), ctypes.c_uint32, vp, vp,
                                         sz, ctypes.c_int64, vp]
        lib.fp_replay_server.restype = ctypes.c_int
        lib.fp_replay_plain.argtypes = [ctypes.POINTER(ReplayBody), ctypes.c_uint32, vp, vp, sz,
                                        ctypes.c_int64, ctypes.c_char, vp, vp]
        lib.fp_replay_plain.restype = ctypes.c_int
        lib.fp_test_arm_stalled_lookback.argtypes = [vp, ctypes.c_uint64]
        lib.fp_test_arm_stalled_lookback.restype = ctypes.c_int
        lib.fp_strerror.argtypes = [ctypes.c_int]
        lib.fp_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().fp_strerror(code).decode()
    except Exception:  # library not loadable: describe the code ourselves
        return "error %d" % code


def check(code: int, where: str) -> None:
    if code != FP_OK:
        raise FpError(code, where)
