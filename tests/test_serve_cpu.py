"""The serving scheduler's logic on the CPU: tests/serve_core_check.cpp
drives paper_1612_04003_gb300/csrc/ca_serve_core.h with a fake executor
(FIFO admission, the footprint bound at every start, releases, rejections,
latency statistics); tests/batch_plan_check.cpp checks the work plan of a
shared launch over uneven instances."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("g++") is None, reason="no g++")
def test_scheduler_core(tmp_path):
    exe = tmp_path / "serve_core_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-pthread", "-I",
                    os.path.join(ROOT, "paper_1612_04003_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "serve_core_check.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr


@pytest.mark.skipif(shutil.which("g++") is None, reason="no g++")
def test_shared_launch_plan(tmp_path):
    """The work plan of a shared Gram launch over uneven instances
    (paper_1612_04003_gb300/csrc/ca_batch_plan.h): coverage of every atom,
    one partial slot per unit, contiguous stretches, balance within one atom."""
    exe = tmp_path / "batch_plan_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I",
                    os.path.join(ROOT, "paper_1612_04003_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "batch_plan_check.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ALL OK" in r.stdout, r.stdout + r.stderr
