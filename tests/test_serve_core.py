"""Host-only tests of the serving loop's core (admission, continuous batching, ticket API,
failure paths, trace replay): serve_core_test.cpp is compiled with the host compiler against the
library's serve_core.h and run with a fake executor, so no GPU is needed."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2005_11547_gb300", "csrc")


def test_serve_core_host_logic():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "serve_core_test")
        r = subprocess.run([cxx, "-std=c++17", "-O1", "-pthread", "-Wall", "-Werror", "-I", CSRC,
                            os.path.join(HERE, "serve_core_test.cpp"), "-o", exe],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and "ALL PASS" in r.stdout, r.stdout + r.stderr
