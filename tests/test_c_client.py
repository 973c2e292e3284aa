"""The C ABI from plain C: a C99 program that includes only include/g3gemm.h
compiles with -Wall -Wextra -pedantic, links only libg3gemm.so and runs its
device-independent checks (argument validation, status strings, the
generated family, the planner).  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2310_20347_gb300")


def test_c_client_builds_and_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    so = os.path.join(PKG, "libg3gemm.so")
    if not os.path.exists(so):
        pytest.skip("libg3gemm.so not built")
    exe = str(tmp_path / "abi_client")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c_client", "abi_client.c"),
           "-o", exe, "-L", PKG, "-lg3gemm", "-Wl,-rpath," + PKG]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "abi client ok" in r.stdout
