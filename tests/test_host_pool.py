"""Host logic without a GPU: the library's host worker pool (mesh ingest runs its
parallel passes on it) gives every job of a call to exactly one thread and
returns only when all have run, with one caller and with several host threads
calling at once (a second caller runs its own jobs alone)."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2108_10481_gb300", "csrc")


def test_host_pool_runs_every_job_once():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "host_pool_driver")
        subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", SRC,
                        os.path.join(ROOT, "tests", "host_pool_driver.cpp"), "-o", exe], check=True, timeout=300)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "single caller 0 bad, concurrent callers 0 bad" in r.stdout
