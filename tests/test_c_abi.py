"""The boundary is plain C: a C99 program that includes include/lift.h,
links the library and calls its host-only entry points builds with
-Wall -Werror and runs without a GPU."""
import os
import shutil
import subprocess

import pytest

from paper_1502_02389_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_client_builds_and_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    build.build()
    lib_dir = os.path.join(ROOT, "paper_1502_02389_gb300")
    exe = str(tmp_path / "abi_client")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client", "abi_client.c"),
                    "-o", exe, os.path.join(lib_dir, "liftblas.so"),
                    "-Wl,-rpath," + lib_dir], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    assert "fixed dot pick dot_" in out and out.strip().endswith("ok")
    assert "gemv features" in out and "status" in out
