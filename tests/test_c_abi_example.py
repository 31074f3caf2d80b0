"""The header is plain C: a C11 program (tests/c_abi_example.c) compiles against it with
-Wall -Werror and links against the library; on a GPU it sketches a batch through the
host-buffer entry and prints the oracle's keys."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def example():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    import paper_2005_11547_gb300 as pkg
    lib = pkg.build()
    tmp = tempfile.mkdtemp()
    exe = os.path.join(tmp, "c_abi_example")
    r = subprocess.run([cc, "-std=c11", "-O1", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        os.path.join(HERE, "c_abi_example.c"), lib, "-Wl,-rpath," + os.path.dirname(lib),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    yield exe
    shutil.rmtree(tmp, ignore_errors=True)


def test_compiles_and_links_as_c(example):
    assert os.path.exists(example)


@pytest.mark.gpu
def test_runs_and_matches_oracle(example, oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b = workloads.random_sets(50, 0, 120, 1 << 22, seed=4)
    lines = [str(b.n_sets), " ".join(str(int(v)) for v in b.indptr)]
    lines += [f"{int(i)} {float(w)!r}" for i, w in zip(b.indices, b.weights)]
    r = subprocess.run([example, "64"], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    got = np.array([int(x, 16) for x in r.stdout.split()], dtype=np.uint64).reshape(b.n_sets, 64)
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1)
    assert np.array_equal(got, exp)
