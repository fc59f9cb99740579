"""The request server's device-memory allocator (host C++, no GPU): built
here with the host compiler and checked against a bitmap model."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def arena_check(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_check")
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-Werror", "-o", exe,
                    os.path.join(HERE, "native", "arena_check.cpp")], check=True)
    return exe


@pytest.mark.parametrize("cap,steps,seed", [(64, 20000, 1), (4096, 60000, 2), (1000, 60000, 3),
                                            (1, 1000, 4)])
def test_arena_matches_bitmap_model(arena_check, cap, steps, seed):
    r = subprocess.run([arena_check, str(cap), str(steps), str(seed)], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr


def test_arena_under_sanitizers(tmp_path):
    """The same model check built with AddressSanitizer and
    UndefinedBehaviorSanitizer."""
    cxx = shutil.which("g++")
    if not cxx:
        pytest.skip("no g++")
    exe = str(tmp_path / "arena_check_san")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined",
                        "-fno-sanitize-recover=undefined", "-Wall", "-Werror", "-o", exe,
                        os.path.join(HERE, "native", "arena_check.cpp")],
                       capture_output=True, text=True)
    if r.returncode:
        pytest.skip("sanitizer runtime not available: " + r.stderr.strip()[:200])
    for cap, steps, seed in ((64, 20000, 1), (4096, 60000, 2), (1, 1000, 4)):
        r = subprocess.run([exe, str(cap), str(steps), str(seed)], capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
        assert "runtime error" not in r.stderr, r.stderr
