"""The wide-range kernel's exact integer arithmetic, run on the host: dm_wide.cu's geometry,
rank-cut, code and walk helpers compiled for the CPU and driven one element at a time
(tests/wide_host_check.cu) give the wide oracle's keys and status codes, for every norm of
Table 1, weights spanning 2^{+-300} in a set, repeated ids, subnormal weights, zero rows and
the range errors, with the default first limit and with one that needs retry passes."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import workloads

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2005_11547_gb300", "csrc")


def batch(seed):
    rng = np.random.default_rng(seed)
    rows = []
    for norm in [1.0, 2.0 ** 64, 2.0 ** -64, 2.0 ** 512, 2.0 ** -512, 3.7, 2.0 ** -30, 2.0 ** 200]:
        for _ in range(3):
            rows.append(workloads.wide_set(rng, int(rng.integers(1, 24)), norm))
    for _ in range(5):
        m = int(rng.integers(2, 12))
        rows.append((workloads.wide_ids(rng, m), 2.0 ** rng.uniform(-300, 300, size=m)))
    rows += [(np.array([5, 5, 9], np.uint64), np.array([0.5, 0.25, 0.0])),
             (np.array([2 ** 64 - 1, 3], np.uint64), np.array([5e-324, 1.0])),
             (np.array([7], np.uint64), np.array([0.0])),
             (np.array([], np.uint64), np.array([])),
             (np.array([1, 2], np.uint64), np.array([2.0 ** 959, 2.0 ** 958])),
             (np.array([1, 2], np.uint64), np.array([2.0 ** -991, 1e-310])),
             (np.array([1, 2], np.uint64), np.array([0.5, np.nan])),
             (np.array([1, 2], np.uint64), np.array([2.0 ** 961, 1.0]))]
    return workloads.wide_csr(rows)


@pytest.fixture(scope="module")
def host_lib():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("no nvcc")
    tmp = tempfile.mkdtemp()
    so = os.path.join(tmp, "libwidehost.so")
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-Xcompiler", "-fPIC", "-shared",
                        os.path.join(HERE, "wide_host_check.cu"), "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(so)
    P = ctypes.c_void_p
    lib.wide_host_sketch.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_double, P, P, P]
    yield lib
    shutil.rmtree(tmp, ignore_errors=True)


@pytest.mark.parametrize("k,phi0", [(7, 1.25), (64, 0.3), (256, 1.25)])
def test_host_walk_matches_oracle(host_lib, k, phi0):
    from oracle import poisson_thresholds, t_of_k, wide
    b = batch(k)
    T = np.ascontiguousarray(poisson_thresholds())
    ip = np.ascontiguousarray(b.indptr, np.int64)
    ix = np.ascontiguousarray(b.indices, np.uint64)
    w = np.ascontiguousarray(b.weights, np.float64)
    out = np.zeros((b.n_sets, k), np.uint64)
    st = np.zeros(b.n_sets, np.int32)
    host_lib.wide_host_sketch(ip.ctypes.data, ix.ctypes.data, w.ctypes.data, b.n_sets, k, t_of_k(k), 13, phi0,
                              T.ctypes.data, out.ctypes.data, st.ctypes.data)
    exp, est = wide.sketch(b.indptr, b.indices, b.weights, k, 13)
    assert np.array_equal(st, est)
    assert list(est[-4:]) == [0, 5, 1, 5]            # in range, tiny row, NaN, 2^961
    assert np.array_equal(out, exp)
