"""Host logic of the library on the CPU: the first-fit arena allocator with
its fault injector (every out-of-memory position unwinds without leaking)
and the server's admission queue (admission waits for memory, a request
that can never fit is rejected, cancellation only while waiting).  The
checks are a small C++ driver over the library's own header, built here
with the system compiler; no GPU is involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_logic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = tmp_path / "host_logic_test"
    src = os.path.join(ROOT, "tests", "host", "host_logic_test.cpp")
    inc = os.path.join(ROOT, "paper_2104_14447_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", inc, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert "host logic ok" in r.stdout
