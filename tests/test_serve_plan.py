"""Host-only planning of the serving engine, checked on the CPU: the arena
ring (including a ring that is exactly full after wrapping) and the batch
planner, whose parts must each fit an empty arena so that the queue always
drains. The planning header has no CUDA in it; a small C++ program that
includes it is built with the host compiler and run."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


@pytest.mark.timeout(300)
def test_serve_plan_checks(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "serve_plan_check")
    csrc = os.path.join(ROOT, "paper_1910_05109_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", csrc,
                    os.path.join(ROOT, "tests", "serve_plan_check.cpp"), "-o", exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr
    assert "passed" in r.stdout
