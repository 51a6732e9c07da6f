"""The C ABI from plain C, without a GPU: include/b64gpu.h compiles as C99
with warnings as errors, and a C program linked against libb64gpu.so gets
the documented results from the entry points that need no device."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT


@pytest.mark.timeout(600)
def test_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1910_05109_gb300 import build, binding
    build.build()
    libdir = os.path.dirname(binding.LIB_PATH)
    exe = str(tmp_path / "abi_c_check")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_c_check.c"),
                    "-L", libdir, "-l:libb64gpu.so", f"-Wl,-rpath,{libdir}", "-o", exe],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert "passed" in r.stdout
