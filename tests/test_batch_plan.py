"""CPU: the batched form's plan (csrc/batch_plan.h).

The plan is plain C++ used by lra_batch_create and by this check: a g++-built
harness (tests/cpp/batch_plan_check.cpp) checks on fixed and 500 random batches
that problems run largest first with ties in the caller's order, that each
problem's block cap is ceil(min(m, n) / 2b) (or max_blocks), that its buffers
sit in the pool on 256-byte boundaries without overlap, and that every tile
list covers each problem's rows or columns exactly once, in internal order.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_plan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path / "batch_plan_check")
    src = os.path.join(ROOT, "tests", "cpp", "batch_plan_check.cpp")
    inc = os.path.join(ROOT, "paper_2506_03859_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", inc, src, "-o", exe], check=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.split() == ["fixed", "ok", "random", "ok"]
