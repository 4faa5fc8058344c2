"""Host check of the digit-pair schedule of the emulated-FP64 products (csrc/oz_schedule.h): a
C++ program (tests/oz_schedule_check.cpp) plays the schedule as the product kernel reads it, in
exact integer arithmetic beside FP32, for K from 64 to the longest single launch.  No GPU."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_oz_schedule_host_check(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "oz_schedule_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2104_14186_gb300", "csrc"),
                    os.path.join(HERE, "oz_schedule_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
