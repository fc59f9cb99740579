#!/usr/bin/env python
"""Throughput of bulk decimal-text -> binary64 parsing on one GB300 (or N).

One step = one parse of the bulk mixed workload: 10,000,000 newline-separated
numbers (about 188 MB of text; 40% uniform [0,1) at 17 significant digits,
30% coordinates with 12-16 fractional digits, 20% integers in [0, 2^63),
10% d.ddddE+-xxx with exponents in [-340, 320]) through fp_parse_f64, with
the text already resident in device memory.  The whole-job value is GB/s of
input text; `e2e` repeats the measurement through fp_parse_f64_host with the
host<->device copies inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank parses its own independently seeded shard (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
`--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import collections
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GB/s of decimal text parsed to binary64 (bit-exact); p50/p99 request latency"
UNIT = "GB/s"
WORKLOAD = ("bulk mixed text, 10M numbers newline-separated: 40% uniform [0,1) at 17 "
            "significant digits, 30% coordinates (lat/lon, 12-16 fractional digits), 20% "
            "integers in [0,2^63), 10% d.ddddE+-xxx with exponents in [-340,320]")
UNIFORM_WORKLOAD = ("uniform: 10,000 doubles uniform in [0,1) printed with %.17g, newline-separated "
                    "(about 190 KB), one buffer")
HARD_WORKLOAD = ("hard cases, 1M strings: 50% with 20-800 significant digits, 30% exact midpoints "
                 "between adjacent doubles in full decimal (exact, +1, -1 in the last digit), 20% "
                 "subnormal and near-DBL_MAX values with 17-25 digits")
FALLBACK_HBM_GBS = 6800.0
L2_BYTES = 129 * 1000 * 1000
def launches_per_call(stats) -> int:
    """Our kernels per parse call: the parse and fallback kernels, and the
    one-block separator the library queues between them when the stream's
    calls have fallback work (so on every timed call of such a workload)."""
    return 3 if stats.get("fallback", 0) > 0 else 2


# end-to-end timings: rounds per line, the median reported
E2E_ROUNDS = 3
# how kernel_ms is measured (the value is the sample interval)
KERNEL_TIMING = ("CUDA events recorded by the library on the call's stream around the kernels of "
                 "every %d-th call of the timed region; the mean over those calls")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def shard_seed(base: int, rank: int) -> int:
    """Seed of rank's shard: every rank parses its own, independent input."""
    return base + 1000 * rank


def max_over_ranks(dist, x: float, device) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's);
    x itself when not distributed."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world: int, bytes_per_rank: int, steps: int, max_ms: float) -> float:
    """Whole-job GB/s: every rank's bytes over the slowest rank's time."""
    return world * bytes_per_rank * steps / (max_ms / 1e3) / 1e9


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


PARSE_KERNEL_SOURCES = ("fp_parse_kernel.cu", "fp_parse_kernel.cuh", "fp_device.cuh",
                        "fp_sync.cuh", "fp_types.cuh", "pow5_table.inc")


def _code_only(src: bytes) -> bytes:
    """C/C++ source with comments and blank lines removed (a comment edit
    does not change the compiled kernel)."""
    import re
    text = src.decode("utf-8", "replace")
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    lines = [ln.rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln.strip()).encode()


def kernel_source_sha(read=None) -> str:
    """Hash of the code (comments removed) the parse kernel is compiled from."""
    d = os.path.join(ROOT, "paper_2101_11408_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(d, name), "rb") as f:
                return f.read()
    h = hashlib.sha256()
    for name in PARSE_KERNEL_SOURCES:
        h.update(name.encode() + b"\0" + _code_only(read(name)))
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch from a committed ncu summary, when that summary
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "%s_bulk_mixed_10m.md" % kernel)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                v = v.strip()
                if v.startswith("`"):
                    v = v[1:].split("`", 1)[0]
                else:
                    v = v.split(" ", 1)[0] if v else v
                vals[k.strip()] = v
    if vals.get("source_sha") != kernel_source_sha():
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cut_at_line(text: bytes, nbytes: int) -> bytes:
    if nbytes >= len(text):
        return text
    k = text.rfind(b"\n", 0, nbytes)
    return text[:k] if k > 0 else text[:nbytes]


def oracle_time(sample: bytes, threads: int, f32: bool = False, delim: bytes = b"\n",
                grammar: int = 0) -> float:
    import oracle
    t = time.perf_counter()
    oracle.parse_buffer(sample, delim, nthreads=threads, f32=f32, grammar=grammar)
    return time.perf_counter() - t


def cpu_baseline(text: bytes, kind: str = "bulk", seconds: float = 10.0, f32: bool = False,
                 delim: bytes = b"\n", grammar: int = 0) -> dict:
    """The oracle on every host core, on a prefix of the workload sized for
    about `seconds` of work (from a 1 MB calibration), repeated when the
    whole text takes less."""
    cores = os.cpu_count() or 1
    calib = cut_at_line(text, 1 << 20)
    rate = len(calib) / oracle_time(calib, cores, f32, delim, grammar)
    sample = cut_at_line(text, int(min(64 << 20, max(1 << 20, rate * seconds))))
    passes = max(1, int(rate * seconds / max(len(sample), 1) / 4))
    t = time.perf_counter()
    for _ in range(passes):
        oracle_time(sample, cores, f32, delim, grammar)
    dt = time.perf_counter() - t
    base = {"value": passes * len(sample) / dt / 1e9, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "first %d bytes (%.2f MB, cut at a line break) of the %s workload, %d "
                      "pass(es), %d threads, %.2f s" % (len(sample), len(sample) / 1e6, kind,
                                                      passes, cores, dt)}
    if not f32 and grammar == 0 and delim == b"\n":
        base["context"] = {"glibc_strtod": strtod_context(sample, cores)}
    return base


def strtod_context(sample: bytes, cores: int, seconds: float = 1.0) -> dict:
    """The C library's strtod on the same sample and threads (context beside
    the oracle: the paper's comparison point; correctly rounded in glibc)."""
    from oracle import context
    n, sec = context.strtod_buffer(sample, b"\n", cores)
    passes = max(1, int(seconds / max(sec, 1e-6)))
    total = 0.0
    for _ in range(passes):
        total += context.strtod_buffer(sample, b"\n", cores)[1]
    return {"value": passes * len(sample) / total / 1e9, "unit": UNIT, "threads": cores,
            "mfloats_per_s": passes * n / total / 1e6, "passes": passes}


def run_reference(args, world, rank) -> None:
    """The oracle on the host cores, bounded samples of the same workload."""
    if rank != 0:
        return
    from paper_2101_11408_gb300 import workloads
    cores = os.cpu_count() or 1
    kind = args.workload if args.workload in ("uniform", "hard") else "bulk"
    gen, n_default, wl_desc, sid = {
        "uniform": (workloads.uniform_text, 10_000, UNIFORM_WORKLOAD, 1),
        "bulk": (workloads.bulk_mixed_text, 10_000_000, WORKLOAD, 2),
        "hard": (workloads.hard_case_text, 1_000_000, HARD_WORKLOAD, 3)}[kind]
    n = args.n or n_default
    text = gen(n, workloads.SEED_BASE + sid)
    calib = cut_at_line(text, 4 << 20)
    rate = len(calib) / oracle_time(calib, cores)
    per_step = int(min(64 << 20, max(1 << 20, rate * args.reference_seconds /
                                     max(1, args.steps + args.warmup))))
    sample = cut_at_line(text, per_step)
    for _ in range(args.warmup):
        oracle_time(sample, cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_time(sample, cores)
    dt = time.perf_counter() - t
    value = len(sample) * args.steps / dt / 1e9
    desc = ("oracle (exact big-number C parser) on %d host threads; each step parses the "
            "first %d bytes (cut at a line break) of the %s workload" % (cores, len(sample), kind))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": {"workload": wl_desc, "numbers": n,
                                        "text_bytes": len(text)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(args, world, rank, dist) -> None:
    import torch

    import paper_2101_11408_gb300 as fp
    from paper_2101_11408_gb300 import workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fp._lib.load()
    kind = args.workload
    seed = shard_seed(workloads.SEED_BASE + {"uniform": 1, "bulk": 2, "hard": 3}[kind], rank)
    gen = {"uniform": workloads.uniform_text, "bulk": workloads.bulk_mixed_text,
           "hard": workloads.hard_case_text}[kind]
    n_default = {"uniform": 10_000, "bulk": 10_000_000, "hard": 1_000_000}[kind]
    desc = {"uniform": UNIFORM_WORKLOAD, "bulk": WORKLOAD, "hard": HARD_WORKLOAD}[kind]
    # a small input sits in L2: flush it between steps and time each step alone
    flush = kind == "uniform"
    t = time.perf_counter()
    text = gen(args.n or n_default, seed)
    log("rank %d: generated %d bytes in %.1f s" % (rank, len(text), time.perf_counter() - t))
    B = len(text)
    host_text = torch.frombuffer(bytearray(text), dtype=torch.uint8)
    d_text = host_text.to(dev)
    f32 = args.format == "f32"
    out = torch.empty(B, dtype=torch.float32 if f32 else torch.float64, device=dev)
    parse_into = fp.parse_f32_into if f32 else fp.parse_f64_into
    vbytes = 4 if f32 else 8  # bytes of one result value
    st = torch.empty(B, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # one untimed parse, checked against the oracle (the whole text, up to
    # --check-mb MB of whole lines)
    parse_into(d_text, out, st, cnt, stream=stream)
    torch.cuda.synchronize()
    N = int(cnt.item())
    check_fields = 0
    if rank == 0 and not args.skip_check:
        import oracle
        prefix = cut_at_line(text, args.check_mb << 20)
        rb, rs = oracle.parse_buffer(prefix, f32=f32)
        got = out[:rb.size].cpu().numpy().view(np.uint32 if f32 else np.uint64)
        gst = st[:rb.size].cpu().numpy()
        if not (np.array_equal(got, rb) and np.array_equal(gst, rs)):
            raise SystemExit("bench: GPU output differs from the oracle")
        check_fields = int(rb.size)
    if fp.get_error():
        raise SystemExit("bench: device error flag set")

    sampler = ClockSampler(local).start() if rank == 0 else None
    for _ in range(args.warmup):
        parse_into(d_text, out, st, cnt, stream=stream)
    # keep the GPU busy for a second before timing so the clock samples
    # describe the same steady state as the timed steps
    t_end = time.perf_counter() + args.clock_settle
    while time.perf_counter() < t_end:
        for _ in range(20):
            parse_into(d_text, out, st, cnt, stream=stream)
        torch.cuda.synchronize()

    # the library's CUDA events around the kernels of every --kernel-sample-th
    # timed call (an event between two kernels ends their programmatic
    # overlap, so timing every call would slow every step a little)
    fp.timing_enable(True, every=args.kernel_sample)
    fp.timing_read(stream)  # reset the sums
    s_before = fp.stats(reset=True, stream=stream)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ms = []
    if flush:
        scrub = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for a, b in evs:
            scrub.fill_(1)  # evict the text and results from L2, outside the timed pair
            a.record(stream)
            parse_into(d_text, out, st, cnt, stream=stream)
            b.record(stream)
        torch.cuda.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        elapsed_ms = sum(step_ms)
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            parse_into(d_text, out, st, cnt, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        elapsed_ms = e0.elapsed_time(e1)
    if dist is not None:
        dist.barrier()
    kt = fp.timing_read(stream)
    fp.timing_enable(False)
    # path counters of the timed calls only (the end-to-end calls below run
    # on the same stream)
    s = fp.stats(reset=True, stream=stream)
    clocks = sampler.stop() if sampler else None
    if dist is not None:
        elapsed_ms = max_over_ranks(dist, elapsed_ms, dev)
    value = whole_job_gbs(world, B, args.steps, elapsed_ms)

    # end to end: host text -> device, parse, results -> host, every step
    e2e = None
    if not args.skip_e2e and not f32:
        h_text = host_text.pin_memory()
        h_out = torch.empty(B, dtype=torch.float64).pin_memory()
        h_st = torch.empty(B, dtype=torch.uint8).pin_memory()
        # a text below 4 MB is timed over 1000 calls or more, tens of
        # milliseconds on the host clock (20 calls of a 0.2 MB text last under
        # a millisecond)
        steps = min(args.steps, args.e2e_steps) if B >= (4 << 20) else max(args.e2e_steps, 1000)
        for _ in range(min(args.warmup, 3)):
            fp.parse_f64_host_into(h_text, h_out, h_st, stream=stream)
        if dist is not None:
            dist.barrier()
        # E2E_ROUNDS timed rounds of `steps` calls each; the value is the
        # median round (the link and the host are shared with other jobs, so
        # one round can be disturbed)
        rounds = []
        n_host = 0
        for _ in range(E2E_ROUNDS):
            t = time.perf_counter()
            for _ in range(steps):
                n_host = fp.parse_f64_host_into(h_text, h_out, h_st, stream=stream)
            dt = time.perf_counter() - t
            if dist is not None:
                dt = max_over_ranks(dist, dt, dev)
            rounds.append(world * B * steps / dt / 1e9)
        assert n_host == N
        if rank == 0 and check_fields:
            assert np.array_equal(h_out[:check_fields].numpy().view(np.uint64),
                                  out[:check_fields].cpu().numpy().view(np.uint64))
        e2e = {"value": float(np.median(rounds)), "unit": UNIT,
               "h2d_bytes_per_step": B, "d2h_bytes_per_step": 9 * N + 8, "steps": steps,
               "rounds": E2E_ROUNDS, "rounds_GBps": [round(r, 1) for r in rounds],
               "api": "fp_parse_f64_host (pinned host buffers)"}

    if rank != 0:
        return
    peak, peak_kind = measured_hbm_peak()
    alg_bytes = B + (vbytes + 1) * N
    parse_ms = kt["parse_ms"] / max(kt["calls"], 1)
    fb_ms = kt["fallback_ms"] / max(kt["calls"], 1)
    achieved = alg_bytes / (parse_ms / 1e3) / 1e9
    traffic = profiled_traffic("parse_kernel") if kind == "bulk" and not f32 else None
    cfg = fp.get_config()
    l2 = ("no flush: each step reads %.0f MB of text and writes %.0f MB of results, more than "
          "the %.0f MB L2" % (B / 1e6, 9 * N / 1e6, L2_BYTES / 1e6))
    if flush:
        l2 = ("flushed: a %.0f MB device buffer is written before every step, outside that "
              "step's event pair" % (2 * L2_BYTES / 1e6))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32" if f32 else "u64", "data": "synthetic",
        "config": {"workload": desc, "numbers": N, "text_bytes": B,
                   "format": "binary32" if f32 else "binary64",
                   "mfloats_per_s": world * N * args.steps / (elapsed_ms / 1e3) / 1e6,
                   "l2": l2,
                   "parallelism": "replicas: one independent shard per GPU",
                   "chunk_bytes": cfg["chunk_bytes"], "ctas_per_sm": cfg["ctas_per_sm"],
                   "checked_fields": check_fields},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "parse_kernel (fused index+parse+Algorithm 1)",
                     "kernel_ms": parse_ms, "fallback_kernel_ms": fb_ms,
                     "kernel_calls_timed": kt["calls"],
                     "kernel_timing": KERNEL_TIMING % args.kernel_sample,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs copy test)"},
        "gpu_launches": launches_per_call(s) * args.steps,
        "clocks": clocks,
        "path_counts_per_step": {k: s[k] // max(s["calls"], 1) for k in (
            "fields", "one_multiply", "two_multiplies", "general_tokenizer", "long_fields",
            "long_settled", "fallback", "fallback_bignum")},
    }
    if step_ms:
        line["us_per_call"] = {"median": 1e3 * statistics.median(step_ms),
                               "p99": 1e3 * float(np.percentile(step_ms, 99)),
                               "min": 1e3 * min(step_ms)}
    if kind == "hard":
        fb = s["fallback"] // max(s["calls"], 1)
        line["fallback"] = {"rate": fb / max(N, 1), "items_per_step": fb,
                            "items_per_s": fb / (fb_ms / 1e3) if fb_ms > 0 else None,
                            "kernel_ms": fb_ms,
                            "long_field_rate": (s["long_fields"] // max(s["calls"], 1)) / max(N, 1)}
    if e2e:
        line["e2e"] = e2e
    if not args.skip_baseline:
        line["cpu_baseline"] = cpu_baseline(text, kind, f32=f32)
    return line


EXT_WORKLOADS = {
    "json": ("JSON numbers: the bulk mixed text (10M numbers newline-separated, every one a valid "
             "JSON number) under the JSON number grammar (fp_parse_ex)"),
    "hex": ("hexadecimal floats, 10M newline-separated: half float.hex() of uniform [0,1) "
            "doubles, half of random finite binary64 bit patterns of either sign (fp_parse_ex, "
            "hexadecimal grammar)"),
    "columns": ("CSV to columns: 1.25M rows of 8 comma-separated uniform [0,1) %.17g values, "
                "stored column-major, field i at column i mod 8, row i div 8 (fp_parse_ex)"),
}


def run_ext(args, world, rank, dist) -> None:
    """The other grammars and the columnar layout (fp_parse_ex), measured
    like the bulk line: text resident in HBM, larger than L2, K timed calls."""
    import torch

    import paper_2101_11408_gb300 as fp
    from paper_2101_11408_gb300 import workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fp._lib.load()
    kind = args.workload
    n = args.n or 10_000_000
    columns, rows_cap, delim, grammar = 0, 0, b"\n", "decimal"
    if kind == "json":
        text = workloads.bulk_mixed_text(n, shard_seed(workloads.SEED_BASE + 2, rank))
        grammar = "json"
    elif kind == "hex":
        text = workloads.hex_float_text(n, shard_seed(workloads.SEED_BASE + 6, rank))
        grammar = "hex"
    else:
        columns = 8
        rows_cap = n // columns
        text = workloads.csv_columns_text(rows_cap, columns,
                                          shard_seed(workloads.SEED_BASE + 7, rank))
        delim = b","
    gid = {"decimal": 0, "hex": 1, "json": 2}[grammar]
    B = len(text)
    d_text = torch.frombuffer(bytearray(text), dtype=torch.uint8).to(dev)
    cap = columns * rows_cap if columns else B
    out = torch.empty(cap, dtype=torch.float64, device=dev)
    st = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call():
        fp.parse_ex_into(d_text, out, st, cnt, delim, grammar, columns, rows_cap, stream)

    # one untimed call, checked against the oracle (whole lines, up to
    # --check-mb MB)
    call()
    torch.cuda.synchronize()
    N = int(cnt.item())
    check_fields = 0
    if rank == 0 and not args.skip_check:
        import oracle
        prefix = cut_at_line(text, args.check_mb << 20)
        rb, rs = oracle.parse_buffer(prefix, delim, grammar=gid)
        k = rb.size
        if columns:
            i = np.arange(k)
            where = (i % columns) * rows_cap + i // columns  # column-major slots
            got = out.cpu().numpy().view(np.uint64)[where]
            gst = st.cpu().numpy()[where]
        else:
            got = out[:k].cpu().numpy().view(np.uint64)
            gst = st[:k].cpu().numpy()
        if not (np.array_equal(got, rb) and np.array_equal(gst, rs)):
            raise SystemExit("bench: GPU output differs from the oracle")
        check_fields = int(k)
    if fp.get_error():
        raise SystemExit("bench: device error flag set")

    sampler = ClockSampler(local).start() if rank == 0 else None
    for _ in range(args.warmup):
        call()
    t_end = time.perf_counter() + args.clock_settle
    while time.perf_counter() < t_end:
        for _ in range(20):
            call()
        torch.cuda.synchronize()
    fp.timing_enable(True, every=args.kernel_sample)
    fp.timing_read(stream)
    fp.stats(reset=True, stream=stream)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    elapsed_ms = e0.elapsed_time(e1)
    if dist is not None:
        dist.barrier()
    kt = fp.timing_read(stream)
    fp.timing_enable(False)
    s = fp.stats(reset=True, stream=stream)
    clocks = sampler.stop() if sampler else None
    if dist is not None:
        elapsed_ms = max_over_ranks(dist, elapsed_ms, dev)
    if rank != 0:
        return
    value = whole_job_gbs(world, B, args.steps, elapsed_ms)
    peak, peak_kind = measured_hbm_peak()
    alg_bytes = B + 9 * N
    parse_ms = kt["parse_ms"] / max(kt["calls"], 1)
    fb_ms = kt["fallback_ms"] / max(kt["calls"], 1)
    achieved = alg_bytes / (parse_ms / 1e3) / 1e9
    mode = {"json": "MODE_JSON", "hex": "hexadecimal grammar", "columns": "MODE_COLUMNS"}[kind]
    line = {
        "metric": "GB/s of text parsed to binary64 (bit-exact), " + kind, "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": EXT_WORKLOADS[kind], "numbers": N, "text_bytes": B,
                   "grammar": grammar, "columns": columns, "rows_cap": rows_cap,
                   "mfloats_per_s": world * N * args.steps / (elapsed_ms / 1e3) / 1e6,
                   "l2": "no flush: each step reads %.0f MB of text and writes %.0f MB of "
                         "results, more than the %.0f MB L2" % (B / 1e6, 9 * N / 1e6,
                                                                L2_BYTES / 1e6),
                   "parallelism": "replicas: one independent shard per GPU",
                   "checked_fields": check_fields},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "parse_kernel (%s)" % mode, "kernel_ms": parse_ms,
                     "fallback_kernel_ms": fb_ms, "kernel_calls_timed": kt["calls"],
                     "kernel_timing": KERNEL_TIMING % args.kernel_sample,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs copy test)"},
        "gpu_launches": launches_per_call(s) * args.steps,
        "clocks": clocks,
        "path_counts_per_step": {k: s[k] // max(s["calls"], 1) for k in (
            "fields", "one_multiply", "two_multiplies", "general_tokenizer", "long_fields",
            "fallback")},
        "e2e": None,
        "e2e_note": "fp_parse_ex has no host-buffer form; the host-to-host path is "
                    "fp_parse_f64_host (decimal grammar, the default line)",
    }
    if not args.skip_baseline:
        line["cpu_baseline"] = cpu_baseline(text, kind, delim=delim, grammar=gid)
    return line


BATCH_WORKLOAD = ("batched: 4096 independent newline-separated buffers of uniform [0,1) %.17g "
                  "values, sizes lognormal (sigma 2) clipped to [1 KiB, 64 MiB], about 2 GiB in "
                  "total, packed in one allocation with every start alignment mod 16")


def _time_steps(torch, stream, fn, steps: int, warmup: int) -> float:
    """ms per step of fn() on `stream`, CUDA events, after warm-up."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_batch(args, world, rank, dist) -> None:
    """Many uneven buffers in one persistent launch, replayed from a CUDA
    graph, against the same buffers with one launch per buffer."""
    import torch

    import paper_2101_11408_gb300 as fp
    from paper_2101_11408_gb300 import workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fp._lib.load()
    t = time.perf_counter()
    texts = workloads.batch_buffers(args.nbuf, args.batch_bytes,
                                    seed=shard_seed(workloads.SEED_BASE + 4, rank))
    packed, starts = workloads.pack_buffers(texts)
    lens = [len(x) for x in texts]
    B = sum(lens)
    log("rank %d: %d buffers, %d bytes in %.1f s" % (rank, len(texts), B, time.perf_counter() - t))
    h_packed = torch.from_numpy(packed).pin_memory()
    d_packed = h_packed.to(dev)
    views = [d_packed[s:s + n] for s, n in zip(starts, lens)]
    offs = [0]
    for n in lens:
        offs.append(offs[-1] + n)
    cap = max(offs[-1], 1)
    out = torch.empty(cap, dtype=torch.float64, device=dev)
    st = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt = torch.zeros(len(texts), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # autotune the chunk size and blocks per SM on the largest buffer
    big = max(range(len(texts)), key=lambda b: lens[b])
    tuned = fp.autotune(views[big])

    # the per-buffer form writes its own copy of the results, compared below
    out1 = torch.empty(cap, dtype=torch.float64, device=dev)
    st1 = torch.empty(cap, dtype=torch.uint8, device=dev)
    cnt1 = torch.zeros(len(texts), dtype=torch.int64, device=dev)
    cnt1_rows = [cnt1[b:b + 1] for b in range(len(texts))]
    out1_rows = [(out1[offs[b]:offs[b + 1]], st1[offs[b]:offs[b + 1]]) for b in range(len(texts))]

    def per_buffer():
        for b in range(len(texts)):
            o, s_ = out1_rows[b]
            fp.parse_f64_into(views[b], o, s_, cnt1_rows[b], stream=stream)

    plan_g = fp.BatchPlan(views, out, st, offs, cnt, graph=True)
    plan_p = fp.BatchPlan(views, out, st, offs, cnt, graph=False)

    def batch_call():
        fp.parse_f64_batch_into(views, out, st, offs, cnt, stream=stream)

    # parity: graph replay == per-buffer launches (all fields), and the oracle
    # on a sample of buffers
    out.fill_(-1.0)
    plan_g.launch(stream)
    per_buffer()
    torch.cuda.synchronize()
    if fp.get_error():
        raise SystemExit("bench: device error flag set")
    if not torch.equal(cnt, cnt1):
        raise SystemExit("bench: batched field counts differ from per-buffer counts")
    counts = cnt.cpu().tolist()
    mask = torch.zeros(cap, dtype=torch.bool, device=dev)
    for b in range(len(texts)):
        mask[offs[b]:offs[b] + counts[b]] = True
    if not (torch.equal(out.view(torch.int64)[mask], out1.view(torch.int64)[mask])
            and torch.equal(st[mask], st1[mask])):
        raise SystemExit("bench: batched results differ from per-buffer results")
    N = int(sum(counts))
    checked = 0
    if rank == 0 and not args.skip_check:
        import oracle
        rnd = np.random.default_rng(5)
        sample = sorted(set(rnd.choice(len(texts), 48, replace=False).tolist()) | {big})
        for b in sample:
            rb, rs = oracle.parse_buffer(texts[b])
            got = out[offs[b]:offs[b] + counts[b]].cpu().numpy().view(np.uint64)
            if not (rb.size == counts[b] and np.array_equal(got, rb) and
                    np.array_equal(st[offs[b]:offs[b] + counts[b]].cpu().numpy(), rs)):
                raise SystemExit("bench: buffer %d differs from the oracle" % b)
            checked += int(rb.size)

    sampler = ClockSampler(local).start() if rank == 0 else None
    t_end = time.perf_counter() + args.clock_settle
    while time.perf_counter() < t_end:
        plan_g.launch(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_graph = _time_steps(torch, stream, lambda: plan_g.launch(stream), args.steps, args.warmup)
    if dist is not None:
        dist.barrier()
        ms_graph = max_over_ranks(dist, ms_graph, dev)
    clocks = sampler.stop() if sampler else None
    few = max(3, min(args.steps, 10))
    ms_plan = _time_steps(torch, stream, lambda: plan_p.launch(stream), args.steps, args.warmup)
    ms_call = _time_steps(torch, stream, batch_call, few, 3)
    t0 = time.perf_counter()
    ms_per = _time_steps(torch, stream, per_buffer, few, 3)
    wall_per = (time.perf_counter() - t0) / (few + 3) * 1e3

    # end to end, host to host, every step: the buffers in G groups of about
    # equal bytes, one graph-replayed plan per group.  Group g's packed text
    # goes to the device on a copy stream; its plan runs once those bytes
    # have landed and packs its results in buffer order on the device
    # (fp_batch_plan_gather); its total comes back, and exactly that many
    # results go to the host arrays at the running total on a third stream.
    # Copies in, parses and copies out of different groups overlap.
    e2e = None
    if not args.skip_e2e:
        G = max(1, min(args.e2e_groups, len(texts)))
        bounds, acc, target = [0], 0, B / G
        for b in range(len(texts)):
            acc += lens[b]
            if acc >= target * len(bounds) and len(bounds) < G and b + 1 < len(texts):
                bounds.append(b + 1)
        bounds.append(len(texts))
        G = len(bounds) - 1
        plans_e = [fp.BatchPlan(views[a:z], out, st, offs[a:z + 1], cnt[a:z], graph=True)
                   for a, z in zip(bounds, bounds[1:])]
        text_rng = [(starts[a], starts[z - 1] + lens[z - 1]) for a, z in zip(bounds, bounds[1:])]
        h_out = torch.empty(N, dtype=torch.float64).pin_memory()
        h_st = torch.empty(N, dtype=torch.uint8).pin_memory()
        d_pv = torch.empty(cap, dtype=torch.float64, device=dev)
        d_ps = torch.empty(cap, dtype=torch.uint8, device=dev)
        d_tot = torch.empty(G, dtype=torch.int64, device=dev)
        h_tot = torch.empty(G, dtype=torch.int64).pin_memory()
        s_in = torch.cuda.Stream(dev)
        s_out = torch.cuda.Stream(dev)

        def e2e_step():
            start = torch.cuda.Event()
            start.record(stream)
            s_in.wait_event(start)
            s_out.wait_event(start)
            landed, packed_ev = [], []
            with torch.cuda.stream(s_in):  # all groups' text in, back to back
                for x0, x1 in text_rng:
                    d_packed[x0:x1].copy_(h_packed[x0:x1], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(s_in)
                    landed.append(ev)
            for g, (a, z) in enumerate(zip(bounds, bounds[1:])):
                stream.wait_event(landed[g])
                plans_e[g].launch(stream)
                plans_e[g].gather(d_pv[offs[a]:], d_ps[offs[a]:], d_tot[g:g + 1], stream)
                with torch.cuda.stream(stream):
                    h_tot[g:g + 1].copy_(d_tot[g:g + 1], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(stream)
                packed_ev.append(ev)
            n = 0
            for g, (a, z) in enumerate(zip(bounds, bounds[1:])):
                packed_ev[g].synchronize()
                k = int(h_tot[g])
                s_out.wait_event(packed_ev[g])
                with torch.cuda.stream(s_out):
                    h_out[n:n + k].copy_(d_pv[offs[a]:offs[a] + k], non_blocking=True)
                    h_st[n:n + k].copy_(d_ps[offs[a]:offs[a] + k], non_blocking=True)
                n += k
            s_out.synchronize()
            return n

        for _ in range(3):
            e2e_step()
        steps = min(args.steps, args.e2e_steps)
        rounds = []  # median of E2E_ROUNDS timed rounds, as for the single-buffer line
        for _ in range(E2E_ROUNDS):
            t0 = time.perf_counter()
            for _ in range(steps):
                n_e2e = e2e_step()
            rounds.append((time.perf_counter() - t0) / steps)
        dt = float(np.median(rounds))
        # the host results are the buffers' results one after the other
        packed_ref = torch.cat([out1[offs[b]:offs[b] + counts[b]] for b in range(len(texts))])
        packed_st = torch.cat([st1[offs[b]:offs[b] + counts[b]] for b in range(len(texts))])
        if n_e2e != N or not (torch.equal(h_out.view(torch.int64), packed_ref.view(torch.int64).cpu())
                              and torch.equal(h_st, packed_st.cpu())):
            raise SystemExit("bench: host batch results differ from the per-buffer ones")
        for pl in plans_e:
            pl.close()
        e2e = {"value": world * B / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(sum(x1 - x0 for x0, x1 in text_rng)),
               "d2h_bytes_per_step": 9 * N + 8 * G, "steps": steps, "groups": G,
               "rounds": E2E_ROUNDS, "rounds_GBps": [round(world * B / r / 1e9, 1) for r in rounds],
               "api": "per group of buffers (about equal bytes): one host->device copy of its "
                      "packed text, fp_batch_plan_launch (graph) and fp_batch_plan_gather once "
                      "it has landed, a copy of its total, then two copies of exactly that many "
                      "results to the host at the running total; copies in, parses and copies "
                      "out of different groups overlap"}
    if rank != 0:
        return
    peak, peak_kind = measured_hbm_peak()
    alg_bytes = B + 9 * N
    gbs = lambda ms: world * B / (ms / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": gbs(ms_graph), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "buffers": len(texts), "text_bytes": B,
                   "numbers": N, "min_buffer": min(lens), "max_buffer": max(lens),
                   "mfloats_per_s": world * N / (ms_graph / 1e3) / 1e6,
                   "l2": "no flush: each step reads %.0f MB of text, more than the L2" % (B / 1e6),
                   "autotuned": tuned, "checked_fields": checked,
                   "parallelism": "replicas: one independent batch per GPU"},
        "forms": {
            "graph_replay": {"ms": ms_graph, "GB/s": gbs(ms_graph), "launch": "one cudaGraphLaunch"},
            "plan": {"ms": ms_plan, "GB/s": gbs(ms_plan), "launch": "memset + 2 kernels"},
            "batch_call": {"ms": ms_call, "GB/s": gbs(ms_call),
                           "launch": "fp_parse_f64_batch: descriptors built and uploaded per call"},
            "per_buffer": {"ms": ms_per, "GB/s": gbs(ms_per), "host_ms": wall_per,
                           "launch": "%d fp_parse_f64 calls (2 kernels each)" % len(texts)},
        },
        "roofline": {"bound": "hbm", "achieved": alg_bytes / (ms_graph / 1e3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": alg_bytes / (ms_graph / 1e3) / 1e9 / peak,
                     "traffic": None, "kernel": "graph: memset + parse_kernel + fallback_kernel",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs copy test)"},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
    }
    if e2e:
        line["e2e"] = e2e
    return line


SERVE_WORKLOAD = ("serving: Poisson arrivals of CSV requests (8 comma-separated columns of uniform "
                  "[0,1) %.17g values, newline rows), sizes lognormal (median 1 MiB, sigma 1.85) clipped "
                  "to [4 KiB, 256 MiB], admitted under a 40 GB device-memory budget, at 25/50/90% "
                  "of the server's peak offered load")


def _percentile_ms(lat_ns, q):
    return float(np.percentile(np.asarray(lat_ns, dtype=np.float64), q)) / 1e6


def run_serve(args, world, rank, dist) -> None:
    """The request server against the plain per-request path, both fed the
    same Poisson arrival traces of host-memory requests."""
    import ctypes

    import torch

    import paper_2101_11408_gb300 as fp
    from paper_2101_11408_gb300 import workloads

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    lib = fp._lib.load()
    rng = np.random.default_rng(shard_seed(workloads.SEED_BASE + 6, rank))
    R = args.serve_bodies
    sizes = np.clip(np.exp(np.log(1 << 20) + 1.85 * rng.standard_normal(R)), 4 << 10,
                    256 << 20).astype(np.int64)
    t = time.perf_counter()
    pool = workloads.csv_pool()
    bodies = []
    for j in range(R):
        text = workloads.csv_request(int(sizes[j]), workloads.SEED_BASE + 7000 + j, pool)
        a = np.frombuffer(text, dtype=np.uint8)
        fields = int(np.count_nonzero((a == 44) | (a == 10))) + 1  # no empty fields, no trailing separator
        h = torch.frombuffer(bytearray(text), dtype=torch.uint8).pin_memory()
        bodies.append((h, torch.empty(fields, dtype=torch.float64).pin_memory(),
                       torch.empty(fields, dtype=torch.uint8).pin_memory(), fields))
    lens = np.array([b[0].numel() for b in bodies], dtype=np.int64)
    mean_bytes = float(lens.mean())
    mean_fields = float(np.mean([b[3] for b in bodies]))
    log("rank %d: %d request bodies, %.1f MB (mean %.2f MB, max %.1f MB) in %.1f s" % (
        rank, R, lens.sum() / 1e6, mean_bytes / 1e6, lens.max() / 1e6, time.perf_counter() - t))

    srv = fp.Server(device_budget=args.serve_budget, max_batch=args.serve_batch,
                    max_inflight=args.serve_inflight, delim=b",",
                    launch_bytes=args.serve_launch_mb << 20)
    stream = torch.cuda.current_stream()
    cnt = ctypes.c_uint64()

    def plain_one(j):
        h, v, s_, fields = bodies[j]
        rc = lib.fp_parse_f64_host(h.data_ptr(), h.numel(), b",", v.data_ptr(), s_.data_ptr(),
                                   ctypes.byref(cnt), stream.cuda_stream)
        if rc != 0 or cnt.value != fields:
            raise SystemExit("bench: plain path failed (%d, %d fields of %d)" % (rc, cnt.value,
                                                                                fields))

    # The timed traces are replayed by native threads (fp_replay_server /
    # fp_replay_plain), which submit every request at its arrival time; the
    # results of a request go to its body's arrays (requests of the same body
    # write the same values), checked against the body's results after
    # every trace.
    rbodies = (fp._lib.ReplayBody * R)(*[
        fp._lib.ReplayBody(h.data_ptr(), h.numel(), v.data_ptr(), s_.data_ptr(), fields)
        for h, v, s_, fields in bodies])

    def check_bodies(what):
        for j in range(R):
            if not np.array_equal(bodies[j][1].numpy().view(np.uint64), ref_bits[j]):
                raise SystemExit("bench: %s: body %d has wrong results" % (what, j))

    def run_server(order, arr_ns, parts=None):
        """Submit request i at t0 + arr_ns[i]; latency = done - that arrival.
        parts collects the latency's pieces: client lag (arrival -> submit),
        queue (submit -> launch) and service (launch -> done)."""
        n = len(order)
        ordr = np.ascontiguousarray(order, dtype=np.uint32)
        arr = np.ascontiguousarray(arr_ns, dtype=np.int64)
        rec = np.zeros(4 * n, dtype=np.int64)
        l0 = srv.stats()["launches"]
        rc = lib.fp_replay_server(srv._h, rbodies, R, ordr.ctypes.data, arr.ctypes.data, n,
                                  2_000_000, rec.ctypes.data)
        if rc != 0:
            raise SystemExit("bench: server trace failed: %s" % fp._lib.strerror(rc))
        launches = max(srv.stats()["launches"] - l0, 1)
        check_bodies("server trace")
        arrival, submit, launch_t, done = rec.reshape(n, 4).T
        lat = (done - arrival).tolist()
        if parts is not None:
            for name, d in (("client_lag", submit - arrival), ("queue", launch_t - submit),
                            ("service", done - launch_t)):
                parts[name] = {"p50_ms": _percentile_ms(d, 50), "p99_ms": _percentile_ms(d, 99)}
            # latency by request size: below 1 MB and from 1 MB on
            small = lens[ordr] < (1 << 20)
            for name, pick in (("below_1MB", small), ("from_1MB", ~small)):
                d = (done - arrival)[pick]
                if d.size:
                    parts[name] = {"requests": int(d.size), "p50_ms": _percentile_ms(d, 50),
                                   "p99_ms": _percentile_ms(d, 99)}
        span = int(done.max() - arrival.min())
        return lat, span, n / launches

    def run_plain(order, arr_ns):
        n = len(order)
        ordr = np.ascontiguousarray(order, dtype=np.uint32)
        arr = np.ascontiguousarray(arr_ns, dtype=np.int64)
        rec = np.zeros(2 * n, dtype=np.int64)
        rc = lib.fp_replay_plain(rbodies, R, ordr.ctypes.data, arr.ctypes.data, n, 2_000_000,
                                 b",", stream.cuda_stream, rec.ctypes.data)
        if rc != 0:
            raise SystemExit("bench: plain trace failed: %s" % fp._lib.strerror(rc))
        check_bodies("plain trace")
        arrival, done = rec.reshape(n, 2).T
        return (done - arrival).tolist(), int(done.max() - arrival.min())

    def perm_order(n, seed):
        r = np.random.default_rng(seed)
        return np.concatenate([r.permutation(R) for _ in range((n + R - 1) // R)])[:n]

    # correctness: every body once through the server and once alone, against
    # each other, and a sample of bodies against the oracle
    rids0 = [srv.submit(*bodies[j][:3]) for j in range(R)]
    for j in range(R):
        inf = srv.wait(rids0[j])
        if inf["error"] or inf["count"] != bodies[j][3]:
            raise SystemExit("bench: server request for body %d failed: %r" % (j, inf))
    ref_bits = [b[1].numpy().view(np.uint64).copy() for b in bodies]
    for j in range(R):
        plain_one(j)
        if not np.array_equal(bodies[j][1].numpy().view(np.uint64), ref_bits[j]):
            raise SystemExit("bench: body %d differs between the server and the plain path" % j)
    checked = 0
    if rank == 0 and not args.skip_check:
        import oracle
        for j in sorted(range(R), key=lambda j: lens[j])[:: max(1, R // 24)][:24]:
            rb, _ = oracle.parse_buffer(bytes(bodies[j][0].numpy()), b",")
            if not np.array_equal(rb, ref_bits[j]):
                raise SystemExit("bench: body %d differs from the oracle" % j)
            checked += int(rb.size)

    # peak: closed-loop bursts (every arrival at time 0)
    reps = 3
    order = perm_order(R * reps, 11)
    lat, span, _ = run_server(order, np.zeros(len(order)))
    peak_server = float(lens[order].sum()) / (span / 1e9) / 1e9
    t0 = time.perf_counter()
    for j in order[:R]:
        plain_one(int(j))
    peak_plain = float(lens[order[:R]].sum()) / (time.perf_counter() - t0) / 1e9
    log("peak: server %.1f GB/s, plain %.1f GB/s" % (peak_server, peak_plain))

    sampler = ClockSampler(local).start() if rank == 0 else None
    s0 = srv.stats()
    levels = []
    for k, load in enumerate((0.25, 0.5, 0.9)):
        rate = load * peak_server * 1e9 / mean_bytes  # requests per second
        n = int(min(args.serve_max_requests, max(2 * R, rate * args.serve_seconds)))
        r = np.random.default_rng(100 + k)
        arr = np.cumsum(r.exponential(1e9 / rate, size=n))
        arr -= arr[0]
        order = perm_order(n, 200 + k)
        nbytes = float(lens[order].sum())
        parts = {}
        lat_s, span_s, mean_batch = run_server(order, arr, parts)
        lat_p, span_p = run_plain(order, arr)
        levels.append({
            "load": load, "offered_GBps": load * peak_server, "requests": n,
            "seconds": float(arr[-1]) / 1e9,
            "server": {"GBps": nbytes / (span_s / 1e9) / 1e9, "p50_ms": _percentile_ms(lat_s, 50),
                       "p99_ms": _percentile_ms(lat_s, 99), "mean_batch": float(mean_batch),
                       "latency_parts": parts},
            "plain": {"GBps": nbytes / (span_p / 1e9) / 1e9, "p50_ms": _percentile_ms(lat_p, 50),
                      "p99_ms": _percentile_ms(lat_p, 99)},
        })
        log("load %.2f: %r" % (load, levels[-1]))
    s1 = srv.stats()
    clocks = sampler.stop() if sampler else None
    srv.close()
    if rank != 0:
        return
    top = levels[-1]
    line = {
        "metric": METRIC, "value": top["server"]["GBps"], "unit": UNIT, "n_gpus": world,
        "steps": len(levels), "warmup": args.warmup, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "bodies": R, "mean_request_bytes": mean_bytes,
                   "max_request_bytes": int(lens.max()), "device_budget": args.serve_budget,
                   "max_batch": args.serve_batch, "max_inflight": args.serve_inflight,
                   "launch_mb": args.serve_launch_mb or 32,
                   "checked_fields": checked,
                   "l2": "requests stream from host memory; no L2 reuse between requests",
                   "parallelism": "replicas: one independent server per GPU"},
        "p50_ms": top["server"]["p50_ms"], "p99_ms": top["server"]["p99_ms"],
        "peak": {"server_GBps": peak_server, "plain_GBps": peak_plain},
        "levels": levels,
        "e2e": {"value": top["server"]["GBps"], "unit": UNIT,
                "h2d_bytes_per_step": int(mean_bytes), "d2h_bytes_per_step": int(9 * mean_fields),
                "api": "fp_server_submit / fp_server_wait on pinned host buffers: every serving "
                       "number is host to host (a step is one request, sizes are means)"},
        "gpu_launches": 2 * (s1["launches"] - s0["launches"]),
        "server_stats": s1,
        "clocks": clocks,
    }
    return line


def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=0,
                    help="numbers per shard (0: the workload's own size)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--kernel-sample", type=int, default=8,
                    help="time the kernels of every k-th timed call with CUDA events (k >= 1)")
    ap.add_argument("--clock-settle", type=float, default=1.0,
                    help="seconds of untimed steps before the timed region")
    ap.add_argument("--reference-seconds", type=float, default=60.0,
                    help="target duration of the reference arm's timed steps")
    ap.add_argument("--skip-baseline", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--check-mb", type=int, default=512,
                    help="text checked against the oracle before timing (MB of whole lines)")
    ap.add_argument("--no-extras", action="store_true",
                    help="bulk: leave out the hard-case, batched and served sections")
    ap.add_argument("--workload", choices=["bulk", "uniform", "hard", "batch", "serve", "json",
                                           "hex", "columns"],
                    default="bulk",
                    help="bulk: one 10M-number buffer (default); uniform: 10,000 numbers; hard: "
                         "1M hard cases; batch: 4096 uneven buffers; serve: Poisson request "
                         "traces through the request server; json / hex / columns: fp_parse_ex "
                         "under the JSON or hexadecimal grammar, or CSV to column-major")
    ap.add_argument("--serve-bodies", type=int, default=256, help="serve: distinct requests")
    ap.add_argument("--serve-seconds", type=float, default=2.0, help="serve: trace length")
    ap.add_argument("--serve-max-requests", type=int, default=60000)
    ap.add_argument("--serve-budget", type=int, default=40_000_000_000)
    ap.add_argument("--serve-batch", type=int, default=1024)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--serve-launch-mb", type=int, default=0, help="serve: MB per launch (0: 32)")
    ap.add_argument("--format", choices=["f64", "f32"], default="f64",
                    help="bulk/uniform/hard: binary64 (fp_parse_f64) or binary32 (fp_parse_f32)")
    ap.add_argument("--nbuf", type=int, default=4096, help="batch: buffers")
    ap.add_argument("--e2e-groups", type=int, default=8,
                    help="batch: buffer groups of the end-to-end pipeline")
    ap.add_argument("--batch-bytes", type=int, default=2 << 30, help="batch: total text bytes")
    return ap


def _condensed_levels(levels):
    return [{"load": lv["load"], "offered_GBps": lv["offered_GBps"], "requests": lv["requests"],
             "server": {k: lv["server"][k] for k in ("GBps", "p50_ms", "p99_ms", "mean_batch")},
             "plain": lv["plain"]} for lv in levels]


def run_extras(args, world, rank, dist) -> dict:
    """The default line's other configurations, each in its own section: the
    hard cases (fallback rate and throughput), the batched buffers (one
    graph-replayed persistent launch against one launch per buffer) and the
    served requests (the server against the plain per-request path, p50/p99
    at 25/50/90% of the server's peak)."""
    import copy

    import torch

    def sub(workload, **over):
        a = copy.copy(args)
        a.workload = workload
        a.skip_baseline = True
        for k, v in over.items():
            setattr(a, k, v)
        return a

    out = {}
    t = time.perf_counter()
    h = run_ours(sub("hard", e2e_steps=min(args.e2e_steps, 10)), world, rank, dist)
    torch.cuda.empty_cache()
    if h:
        out["hard"] = {k: h[k] for k in ("metric", "value", "unit", "ms_per_step", "roofline",
                                         "fallback", "e2e", "path_counts_per_step", "clocks")
                       if k in h}
        out["hard"]["config"] = {k: h["config"][k] for k in ("workload", "numbers", "text_bytes",
                                                              "mfloats_per_s", "checked_fields")}
        out["hard"]["seconds"] = time.perf_counter() - t
    t = time.perf_counter()
    b = run_batch(sub("batch", e2e_steps=min(args.e2e_steps, 10)), world, rank, dist)
    torch.cuda.empty_cache()
    if b:
        out["batch"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "forms",
                                          "roofline", "e2e", "clocks") if k in b}
        out["batch"]["config"] = {k: b["config"][k] for k in (
            "workload", "buffers", "text_bytes", "numbers", "min_buffer", "max_buffer",
            "mfloats_per_s", "autotuned", "checked_fields")}
        out["batch"]["seconds"] = time.perf_counter() - t
    t = time.perf_counter()
    sv = run_serve(sub("serve", serve_seconds=min(args.serve_seconds, 1.5)), world, rank, dist)
    torch.cuda.empty_cache()
    if sv:
        out["serve"] = {"metric": sv["metric"], "unit": sv["unit"], "p50_ms": sv["p50_ms"],
                        "p99_ms": sv["p99_ms"], "peak": sv["peak"],
                        "levels": _condensed_levels(sv["levels"]), "e2e": sv["e2e"],
                        "clocks": sv.get("clocks"),
                        "config": {k: sv["config"][k] for k in (
                            "workload", "bodies", "mean_request_bytes", "max_request_bytes",
                            "device_budget", "max_batch", "max_inflight", "checked_fields")}}
        out["serve"]["seconds"] = time.perf_counter() - t
    return out


def main() -> None:
    ap = make_parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    line = None
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        line = run_batch(args, world, rank, dist)
    elif args.workload == "serve":
        line = run_serve(args, world, rank, dist)
    elif args.workload in EXT_WORKLOADS:
        line = run_ext(args, world, rank, dist)
    else:
        line = run_ours(args, world, rank, dist)
        # the default line also carries the hard-case, batched and served
        # configurations (one GPU: replicas of those under torchrun would
        # only repeat them)
        if args.workload == "bulk" and not args.no_extras and world == 1:
            import torch
            torch.cuda.empty_cache()
            extras = run_extras(args, world, rank, dist)
            if line is not None:
                line.update(extras)
    if line is not None:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
