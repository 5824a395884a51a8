"""The C ABI from a plain C99 program (no GPU needed): kifmm.h must compile
as C with warnings as errors, and a C caller linked against libkifmm.so
must see the documented answers (tests/c/abi_from_c.c)."""
import os
import shutil
import subprocess

import pytest

from paper_2303_08394_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_08394_gb300 import build
    build.build()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_caller(tmp_path):
    exe = tmp_path / "abi_from_c"
    libdir = os.path.dirname(N.LIB_PATH)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_from_c.c"),
           "-L", libdir, "-l:" + os.path.basename(N.LIB_PATH), "-Wl,-rpath," + libdir,
           "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
