"""CPU: the serving runtime's admission policy (csrc/serve_policy.h).

The policy is plain C++ shared by the library and this check: a g++-built
harness (tests/cpp/serve_policy_check.cpp) drives it through fixed scenarios and
a random trace of 5000 requests and checks that the device-memory budget and
the slot count are never exceeded, that requests start in arrival order
(a large request at the head is not overtaken), that oversize requests are
refused, and that a context kept for the caller holds its bytes but not a slot.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_admission_policy(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "serve_policy_check")
    src = os.path.join(ROOT, "tests", "cpp", "serve_policy_check.cpp")
    inc = os.path.join(ROOT, "paper_2506_03859_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.split() == ["fifo", "ok", "slots", "ok", "kept", "ok", "random", "ok"]
