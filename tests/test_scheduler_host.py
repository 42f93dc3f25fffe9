"""The serving loop's request scheduler (host C++, no CUDA) compiled with g++ and
driven by a fake executor: per-basis FIFO order, concurrency across bases,
admission by the byte budget, refusal of oversized requests, latency percentiles
and draining at shutdown."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_scheduler_host(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "sched_test"
    src = os.path.join(ROOT, "tests", "scheduler_host_test.cpp")
    inc = os.path.join(ROOT, "paper_1903_00548_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-Wall", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr + r.stdout
    assert "passed" in r.stdout
