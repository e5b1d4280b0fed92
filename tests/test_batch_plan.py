"""The host-side batch plan (csrc/lcs_plan.h) checked on CPU: tests/plan_check.cpp, compiled with g++, builds plans
for seeded random batches under every batch configuration and checks their invariants (every pair once, split jobs,
items of one shape that fit a warp, longest first, disjoint and aligned code lists and mask tables, prep order)."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_batch_plan_invariants(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = tmp_path / "plan_check"
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror",
                        "-I", os.path.join(ROOT, "paper_1306_4627_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "plan_check.cpp"), "-o", str(exe)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-3000:]
    assert r.stdout.startswith("ok "), r.stdout
