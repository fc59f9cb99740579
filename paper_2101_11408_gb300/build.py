"""Build the CUDA library in-tree: paper_2101_11408_gb300/_build/libfpparse.so.

Every translation unit is compiled for sm_103a only (-gencode
arch=compute_103a,code=sm_103a), in parallel, and linked with nvcc into one
shared object exporting the C ABI of include/fpparse.h (and the test hooks of
include/fpparse_test.h and the trace replay of include/fpparse_bench.h).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfpparse.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["fp_parse_kernel.cu", "fp_parse_kernel_ext.cu", "fp_fallback_kernel.cu", "fp_api.cu",
           "fp_noalloc.cu", "fp_server.cu", "fp_copy_kernel.cu", "fp_replay.cpp"]
HEADERS = ["fp_device.cuh", "fp_sync.cuh", "fp_types.cuh", "fp_launch.h", "fp_internal.h",
           "fp_parse_kernel.cuh", "fp_copy.h", "fp_arena.h", "pow5_table.inc", "dec_tables.inc",
           os.path.join(INCLUDE, "fpparse.h"), os.path.join(INCLUDE, "fpparse_test.h"),
           os.path.join(INCLUDE, "fpparse_bench.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
                     "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libfpparse")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    for g in ("gen_pow5_table.py", "gen_dec_tables.py"):
        subprocess.run([sys.executable, os.path.join(CSRC, g)], check=True)
    headers = [os.path.join(CSRC, h) if not os.path.isabs(h) else h for h in HEADERS]
    objs, procs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        objs.append(o)
        if force or _stale(o, [s, __file__] + headers):
            cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if ptxas_info else []) + \
                  ["-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose or ptxas_info or p.returncode:
            sys.stdout.write(out)
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    if force or procs or _stale(LIB, objs):
        tmp = LIB + ".%d.tmp" % os.getpid()
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-Xcompiler", "-pthread"]
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
