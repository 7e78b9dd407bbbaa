"""lift_asum_noalloc's argument path, checked without a GPU: the launch
planning it runs before every launch (csrc/noalloc_plan.h) sends an x that
is only 4-byte aligned to 4-byte loads (a 128-bit load there would fault),
keeps the grid within the fixed scratch array, and refuses bad arguments
before any CUDA call."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_noalloc_plan_host_only(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "noalloc_plan_check")
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_1502_02389_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c_client", "noalloc_plan_check.cpp"),
                    "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("all ok")
    assert "FAIL" not in out.stdout
