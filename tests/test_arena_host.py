"""The first-fit arena that carves replica buffers out of the device pool
(host-only C++, compiled with the system compiler)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def arena_check():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    out = os.path.join(HERE, "_build", "arena_check")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", out,
                    os.path.join(HERE, "helpers", "arena_check.cpp")], check=True)
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_arena_first_fit_disjoint_coalescing(arena_check, seed):
    r = subprocess.run([arena_check, str(seed)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("OK")
