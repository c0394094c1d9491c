"""The host worker pool of the plan (paper_2604_00250_gb300/csrc/host_pool.h), built with g++
and run on the CPU: chunk coverage, concurrent submitters, and no pool in a forked child."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_pool(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = tmp_path / "host_pool_check"
    src = os.path.join(ROOT, "tests", "native", "host_pool_check.cpp")
    inc = os.path.join(ROOT, "paper_2604_00250_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O2", "-pthread", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
