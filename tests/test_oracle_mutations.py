"""The oracle's pins must catch plausible mistakes.  Each case plants one mistake in a
temporary copy of oracle/dm_oracle.c (the committed oracle is untouched), builds it, and
checks that the brute-force enumeration or a distributional pin rejects it."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import bruteforce as bf

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "dm_oracle.c")

MUTATIONS = {
    # the rank increment uses delta_nu's power instead of delta_rho's (transposed operand)
    "rank_delta_transposed": ("((((u128)r << 24) | u) << rho)", "((((u128)r << 24) | u) << nu)"),
    # the weight offset W = (2^nu - 1)/t is dropped from the dart weight
    "weight_offset_dropped": ("dy sw = { (p2m1(nu) << (rho + 24)) + ", "dy sw = { "),
    # top weight region skipped (off by one in the region bound)
    "region_bound_off_by_one": ("dy wlo = { p2m1(nu), 0 };", "dy wlo = { p2m1(nu + 1), 0 };"),
    # Poisson inversion reads the wrong threshold
    "poisson_index_shift": ("if (u >= T[n]) x++;", "if (u >= T[n < 11 ? n + 1 : n]) x++;"),
    # one shift of the mixer changed
    "mixer_shift": ("z = (z ^ (z >> 27))", "z = (z ^ (z >> 26))"),
    # the row break compares a doubled row edge, so rows holding kept darts are skipped
    # (the opposite slip, a halved edge, only visits extra rows and changes no output)
    "row_edge_doubled": ("dy cr = { (p2m1(rho) << nu) + ((u128)r << rho), -nu };",
                         "dy cr = { (p2m1(rho) << nu) + ((u128)r << rho), -nu + 1 };"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(mutated)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    P = ctypes.c_void_p
    lib.dmo_sketch.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                               ctypes.c_int64, P, ctypes.c_double, ctypes.c_int32, P, P]
    lib.dmo_sketch.restype = ctypes.c_int
    return lib


def _sketch(lib, oracle_mod, indptr, idx, w, k, seed, work=False):
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    w = np.ascontiguousarray(w, dtype=np.float32)
    n = len(indptr) - 1
    out = np.zeros((n, k), dtype=np.uint64)
    wk = np.zeros((n, 4), dtype=np.int64)
    T = oracle_mod.poisson_thresholds()
    rc = lib.dmo_sketch(P(indptr), P(idx), P(w), n, k, seed, oracle_mod.t_of_k(k), P(T), 1.0, 0,
                        P(out), P(wk))
    return rc, out, wk


def P(a):
    return ctypes.c_void_p(a.ctypes.data)


def _pins_fail(lib, oracle_mod):
    """True when at least one pin rejects the library."""
    T = oracle_mod.poisson_thresholds()
    rng = np.random.default_rng(17)
    # (1) brute force on tiny sets
    for trial in range(25):
        k = int(rng.choice([2, 3, 5]))
        t = oracle_mod.t_of_k(k)
        nnz = int(rng.integers(1, 4))
        idx = np.sort(rng.choice(3000, nnz, replace=False)).astype(np.uint32)
        w = (rng.random(nnz) * 10 ** rng.uniform(-2, 0.5) + 1e-6).astype(np.float32)
        l1 = float(w.astype(np.float64).sum())
        y = max(float(x) * t for x in w)
        nu_box = 0
        while 2 ** (nu_box + 1) - 1 <= y:
            nu_box += 1
        R = 14.0 * k / (t * l1)
        rho_box = 0
        while 2 ** (rho_box + 1) - 1 < R:
            rho_box += 1
        if nnz * (2 ** (nu_box + 1) - 1) * (2 ** (rho_box + 1) - 1) > 20000:
            continue
        rc, out, _ = _sketch(lib, oracle_mod, [0, nnz], idx, w, k, 5)
        if rc:
            return True
        b = bf.sketch(idx, w, k, t, 5, nu_box, rho_box, T)
        if any(b[j] is not None and b[j] != int(out[0, j]) for j in range(k)):
            return True
    # (2) Lemma 1 / Theorem 1 fill probability on k = 64
    import workloads
    bt = workloads.random_sets(1500, 1, 40, 1 << 22, seed=364)
    rc, _, wk = _sketch(lib, oracle_mod, bt.indptr, bt.indices, bt.weights, 64, 5, work=True)
    if rc:
        return True
    p = (1 - math.exp(-331 / 64)) ** 64
    one = int((wk[:, 3] == 1).sum())
    return abs(one - 1500 * p) / math.sqrt(1500 * p * (1 - p)) > 4


def test_unmutated_copy_passes(tmp_path, oracle_mod):
    lib = _build_mutant(tmp_path, "identity", "enum {", "enum {")
    assert not _pins_fail(lib, oracle_mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, oracle_mod, name):
    old, new = MUTATIONS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert _pins_fail(lib, oracle_mod), name
