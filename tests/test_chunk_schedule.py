"""The chunk schedules of bigger mode (host C++: which chunk goes into which
device buffer, leaf chunks and the paper's point chunks), compiled with the
host compiler and checked on simulated calls: no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_chunk_schedules(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "schedule_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I",
                    os.path.join(ROOT, "paper_1512_02831_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "schedule_check.cpp"), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True,
                         timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout
