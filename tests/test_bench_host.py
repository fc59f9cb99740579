"""bench.py's host-side measurement logic, without a GPU: the profile-match
hash of the kernel sources, the traffic taken from a committed profile only
while it matches, the clock-sample summary, line cutting, whole-job GB/s,
and the reference arm's JSON line (the oracle on the host cores)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sources():
    d = os.path.join(ROOT, "paper_2101_11408_gb300", "csrc")
    out = {}
    for name in bench.PARSE_KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            out[name] = f.read()
    return out


def test_source_hash_ignores_comments_and_sees_code():
    src = _sources()
    base = bench.kernel_source_sha(lambda n: src[n])
    assert base == bench.kernel_source_sha()
    commented = dict(src)
    commented["fp_device.cuh"] = (b"// a new comment line\n/* and a block\n comment */\n" +
                                  src["fp_device.cuh"].replace(b"\n", b"  // trailing\n", 3))
    assert bench.kernel_source_sha(lambda n: commented[n]) == base
    changed = dict(src)
    changed["fp_device.cuh"] = src["fp_device.cuh"].replace(b"0x7F7F7F7Fu", b"0x7F7F7F7Eu", 1)
    assert changed["fp_device.cuh"] != src["fp_device.cuh"]
    assert bench.kernel_source_sha(lambda n: changed[n]) != base


def test_profiled_traffic_only_for_the_profiled_sources(monkeypatch, tmp_path):
    # a summary in the committed format, taken on the current sources
    sha = bench.kernel_source_sha()
    (tmp_path / "profiles").mkdir()
    summary = tmp_path / "profiles" / "parse_kernel_bulk_mixed_10m.md"
    summary.write_text("# parse_kernel\n\n- source_sha: `%s` (hash of the sources)\n"
                       "- dram_bytes_per_launch: 244803840\n- duration_us: 252.5 (under ncu)\n"
                       % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_sha", lambda read=None: sha)
    assert bench.profiled_traffic("parse_kernel") == 244803840
    # sources changed since the capture: no traffic figure
    monkeypatch.setattr(bench, "kernel_source_sha", lambda read=None: "0000000000000000")
    assert bench.profiled_traffic("parse_kernel") is None
    assert bench.profiled_traffic("no_such_kernel") is None


def test_clock_summary_reads_samples_and_reasons(tmp_path):
    s = bench.ClockSampler(0)
    s.proc = None
    p = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 540.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 560.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 580.7, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line",
            "0, 1980, 2070, 600.2, 0x0, Not Active, Active, Not Active, Not Active"]
    p.write_text("\n".join(rows) + "\n")

    class Done:  # a finished sampler process
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s.proc, s.path = Done(), str(p)
    r = s.stop()
    assert r["sm_mhz"] == 2062.5 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 4
    assert r["power_w_max"] == 600.2
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert not os.path.exists(p)
    assert bench.ClockSampler(0).stop()["reasons"] == ["nvidia-smi unavailable"]


def test_cut_at_line_and_whole_job_rate():
    text = b"1.5\n22\n333\n4444"
    assert bench.cut_at_line(text, 100) == text
    assert bench.cut_at_line(text, 8) == b"1.5\n22"
    assert bench.cut_at_line(text, 7) == b"1.5\n22"
    assert bench.cut_at_line(text, 6) == b"1.5"
    assert bench.cut_at_line(b"123456", 3) == b"123"
    # 4 ranks x 1e9 bytes x 10 steps in 5 s -> 8 GB/s
    assert bench.whole_job_gbs(4, 10**9, 10, 5000.0) == pytest.approx(8.0)
    assert bench.shard_seed(7, 0) != bench.shard_seed(7, 1)


def test_reference_arm_line():
    """--impl reference: the oracle on the host cores, one JSON line with the
    contract's keys (impl, cpu_baseline, zero-byte e2e)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "uniform", "--steps", "3", "--warmup", "3",
                        "--reference-seconds", "0.3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["steps"] == 3 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_cpu_baseline_fields():
    """The bench line's cpu_baseline: the oracle on all host cores on a
    bounded prefix, with the strtod context for the default grammar only."""
    from paper_2101_11408_gb300 import workloads
    text = workloads.bulk_mixed_text(100000, workloads.SEED_BASE + 81)
    b = bench.cpu_baseline(text, "bulk", seconds=0.3)
    assert b["kind"] == "oracle" and b["unit"] == "GB/s" and b["value"] > 0
    assert b["cores"] == (os.cpu_count() or 1) and "bulk workload" in b["sample"]
    assert b["context"]["glibc_strtod"]["value"] > 0
    j = bench.cpu_baseline(text, "json", seconds=0.2, grammar=2)
    assert j["value"] > 0 and "context" not in j
    c = bench.cpu_baseline(workloads.csv_columns_text(2000, 8, 5), "columns", seconds=0.2,
                           delim=b",")
    assert c["value"] > 0 and "context" not in c


def test_profile_commands_run_committed_files():
    """Every profile summary gives the command that made it; each bench
    invocation there still parses with the bench's current arguments, and
    each ncu line keeps its clocks unlocked."""
    import glob
    import shlex
    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        with open(path) as f:
            text = f.read().replace("\\\n", " ")
        for line in text.splitlines():
            if "ncu " in line:
                assert "--clock-control none" in line, (path, line)
            if "python bench.py" not in line:
                continue
            argv = shlex.split(line.split("python bench.py", 1)[1])
            bench.make_parser().parse_args(argv)  # exits on an unknown flag
            found += 1
    assert found >= 3
