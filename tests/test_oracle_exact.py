"""Exact pins of the oracle (CPU only): values and identities that the paper and the
mathematics fix, and an independent brute-force enumeration of the dart process."""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import bruteforce as bf

U64MAX = np.uint64(2 ** 64 - 1)


# ------------------------------------------------------------------------------------------
# constants
# ------------------------------------------------------------------------------------------
def test_t_values(oracle_mod):
    # Theorem 1's proof fixes t = ceil(k ln k) + k.
    assert oracle_mod.t_of_k(1) == 1
    assert oracle_mod.t_of_k(2) == 4            # 2 ln 2 = 1.386 -> 2, + 2
    assert oracle_mod.t_of_k(64) == 331         # 266.17 -> 267, + 64
    assert oracle_mod.t_of_k(256) == 1676       # 1419.57 -> 1420, + 256
    assert oracle_mod.t_of_k(1024) == 8122      # 7097.83 -> 7098, + 1024
    for k in list(range(2, 300)) + [511, 4096, 8192]:
        assert oracle_mod.t_of_k(k) == math.ceil(k * math.log(k)) + k


def test_poisson_table_is_poisson1_cdf(oracle_mod):
    # Algorithm 1 draws X ~ Poi(1); the table inverts the CDF at 2^-32 resolution.
    T = [int(v) for v in oracle_mod.poisson_thresholds()]
    assert T == sorted(T) and T[-1] < 2 ** 32
    prev = 0
    for n, th in enumerate(T):
        pmf = math.exp(-1.0) / math.factorial(n)
        assert abs((th - prev) / 2 ** 32 - pmf) < 2.5 / 2 ** 32
        prev = th
    # what is left above T[11] is P(X >= 12) rounded to 2^-32
    tail = 1.0 - sum(math.exp(-1.0) / math.factorial(n) for n in range(12))
    assert abs((2 ** 32 - T[-1]) / 2 ** 32 - tail) < 1.5 / 2 ** 32
    assert T[0] == 1580030169                   # ceil(2^32 / e)


def test_mix64_is_splitmix64(oracle_mod):
    # SplitMix64 (Steele, Lea, Flood 2014) started at state 0 outputs these three words.
    g = 0x9E3779B97F4A7C15
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle_mod.mix64(g * n % 2 ** 64) for n in (1, 2, 3)] == expect
    assert [bf.mix64(g * n) for n in (1, 2, 3)] == expect
    rng = np.random.default_rng(3)
    for z in rng.integers(0, 2 ** 63, size=200, dtype=np.int64):
        z = int(z) * 2 + 1
        assert oracle_mod.mix64(z) == bf.mix64(z)


def test_rank_code_rounds_toward_zero():
    for x in [Fraction(1, 3), Fraction(2), Fraction(7, 1024), Fraction(3, 2 ** 40),
              Fraction(2 ** 24 + 1), Fraction(1) - Fraction(1, 2 ** 30)]:
        bits = bf.rz_binary32_bits(x)
        f = np.array([bits], dtype=np.uint32).view(np.float32)[0]
        nxt = np.nextafter(f, np.float32(np.inf))
        assert Fraction(float(f)) <= x < Fraction(float(nxt))


# ------------------------------------------------------------------------------------------
# brute force: the oracle's Algorithm 1 loop == plain enumeration of the dart process
# ------------------------------------------------------------------------------------------
def _boxes(w, k, t):
    l1 = float(np.asarray(w, dtype=np.float64).sum())
    y = max(float(x) * t for x in w)
    nu_box = 0
    while 2 ** (nu_box + 1) - 1 <= y:
        nu_box += 1
    R = 14.0 * k / (t * l1)
    rho_box = 0
    while 2 ** (rho_box + 1) - 1 < R:
        rho_box += 1
    return nu_box, rho_box


def _compare_bruteforce(oracle_mod, idx, w, k, seed):
    t = oracle_mod.t_of_k(k)
    nu_box, rho_box = _boxes(w, k, t)
    areas = len(idx) * (2 ** (nu_box + 1) - 1) * (2 ** (rho_box + 1) - 1)
    if areas > 40000:
        return 0
    o = oracle_mod.sketch(np.array([0, len(idx)]), idx, w, k, seed)[0]
    b = bf.sketch(idx, w, k, t, seed, nu_box, rho_box, oracle_mod.poisson_thresholds())
    n = 0
    for j in range(k):
        if b[j] is not None:
            assert int(o[j]) == b[j], (j, hex(int(o[j])), hex(b[j]))
            n += 1
    return n


def test_bruteforce_random_tiny_sets(oracle_mod):
    rng = np.random.default_rng(11)
    compared = 0
    for trial in range(60):
        k = int(rng.choice([1, 2, 3, 5, 8, 13]))
        nnz = int(rng.integers(1, 5))
        idx = np.sort(rng.choice(5000, nnz, replace=False)).astype(np.uint32)
        scale = 10 ** rng.uniform(-3.0, 1.2)
        w = (rng.random(nnz) * scale + 1e-7).astype(np.float32)
        compared += _compare_bruteforce(oracle_mod, idx, w, k, int(rng.integers(0, 2 ** 62)))
    assert compared > 150


def test_bruteforce_region_edges(oracle_mod):
    # t x_i exactly on a weight-region edge 2^nu - 1 (k = 1: t = 1; k = 2: t = 4), and
    # exactly on a column edge inside a region.
    cases = [(1, [3.0]), (1, [1.0, 3.0]), (1, [7.0, 0.5]), (2, [0.75]), (2, [0.25, 0.75, 1.75]),
             (1, [2.5]), (2, [0.625, 0.375])]
    compared = 0
    for k, ws in cases:
        w = np.array(ws, dtype=np.float32)
        idx = np.arange(len(ws), dtype=np.uint32) * 17 + 3
        for seed in range(6):
            compared += _compare_bruteforce(oracle_mod, idx, w, k, seed)
    assert compared > 20


def test_darthash_dart_set_equals_box(oracle_mod):
    """Algorithm 1 at a fixed rank limit returns exactly the darts of the process that hit x
    and have rank < theta, including theta on region and row edges."""
    T = oracle_mod.poisson_thresholds()
    rng = np.random.default_rng(21)
    for theta in [0.3, 1.0, 1.5, 3.0, 4.25, 7.0, 0.0625]:
        for trial in range(3):
            k = 3
            t = oracle_mod.t_of_k(k)
            nnz = 3
            idx = np.sort(rng.choice(1000, nnz, replace=False)).astype(np.uint32)
            w = (rng.random(nnz) * 0.6 + 0.01).astype(np.float32)
            seed = int(rng.integers(0, 2 ** 40))
            nu_box = 0
            while 2 ** (nu_box + 1) - 1 <= float(w.max()) * t:
                nu_box += 1
            rho_box = 0
            while 2 ** (rho_box + 1) - 1 < theta:
                rho_box += 1
            darts, _ = oracle_mod.darthash(idx, w, t, seed, theta)
            got = sorted((int(d["i"]), int(d["nu"]), int(d["rho"]), int(d["w"]), int(d["r"]),
                          int(d["j"]), (int(d["code"]) << 32) | (int(d["q"]) & 0xFFFFFFFF))
                         for d in darts)
            exp = []
            for i, x in zip(idx, w):
                for rank, key, q, ident in bf.box_darts(int(i), float(x), t, seed, nu_box, rho_box,
                                                        T, with_id=True):
                    if rank < Fraction(float(np.float32(theta))):
                        exp.append((int(i),) + ident + (key,))
            assert got == sorted(exp)


# ------------------------------------------------------------------------------------------
# identities of the definition
# ------------------------------------------------------------------------------------------
def test_subset_of_darts_for_dominated_sets(oracle_mod):
    """Darts are consistent across sets (Section 2): x <= y coordinatewise implies that the
    darts hitting x are a subset of those hitting y."""
    rng = np.random.default_rng(5)
    t = oracle_mod.t_of_k(64)
    for trial in range(20):
        nnz = int(rng.integers(1, 40))
        idx = np.sort(rng.choice(1 << 20, nnz, replace=False)).astype(np.uint32)
        y = (rng.exponential(size=nnz) * 10 ** rng.uniform(-2, 1)).astype(np.float32)
        x = (y * rng.random(nnz).astype(np.float32)).astype(np.float32)
        x[rng.random(nnz) < 0.2] = 0.0
        theta = float(10 ** rng.uniform(-2.5, 0.5))
        dx, _ = oracle_mod.darthash(idx, x, t, 9, theta)
        dy, _ = oracle_mod.darthash(idx, y, t, 9, theta)
        key = lambda d: (int(d["i"]), int(d["nu"]), int(d["rho"]), int(d["w"]), int(d["r"]), int(d["j"]))
        sx, sy = set(map(key, dx)), set(map(key, dy))
        assert sx <= sy
        assert len(sx) <= len(sy)


def test_schedule_and_phi0_invariance(oracle_mod):
    b = workloads.random_sets(120, 1, 60, 1 << 20, seed=77)
    ref = oracle_mod.sketch(b.indptr, b.indices, b.weights, 48, 5)
    for kw in [dict(phi0=2.0), dict(phi0=4.0), dict(phi0=0.3), dict(schedule="step"),
               dict(schedule="step", phi0=3.0)]:
        assert (oracle_mod.sketch(b.indptr, b.indices, b.weights, 48, 5, **kw) == ref).all(), kw


def test_permutation_and_duplicates(oracle_mod):
    rng = np.random.default_rng(8)
    idx = np.sort(rng.choice(1 << 20, 50, replace=False)).astype(np.uint32)
    w = rng.exponential(size=50).astype(np.float32)
    ref = oracle_mod.sketch([0, 50], idx, w, 64, 3)
    p = rng.permutation(50)
    assert (oracle_mod.sketch([0, 50], idx[p], w[p], 64, 3) == ref).all()
    # a duplicated index with a smaller weight changes nothing (union of darts = max weight)
    idx2 = np.concatenate([idx, idx[:10]])
    w2 = np.concatenate([w, w[:10] * np.float32(0.5)]).astype(np.float32)
    assert (oracle_mod.sketch([0, 60], idx2, w2, 64, 3) == ref).all()
    # zero weights are ignored
    idx3 = np.concatenate([idx, np.array([7, 9], dtype=np.uint32)])
    w3 = np.concatenate([w, np.zeros(2, dtype=np.float32)])
    assert (oracle_mod.sketch([0, 52], idx3, w3, 64, 3) == ref).all()


def test_empty_rows_give_sentinel(oracle_mod):
    out = oracle_mod.sketch([0, 0, 3, 3], np.array([1, 2, 3], np.uint32),
                            np.zeros(3, np.float32), 16, 1)
    assert (out == U64MAX).all()


def test_invalid_weights_are_rejected(oracle_mod):
    for bad in [-1.0, float("nan"), float("inf")]:
        with pytest.raises(oracle_mod.OracleError) as e:
            oracle_mod.sketch([0, 2], np.array([1, 2], np.uint32), np.array([0.5, bad], np.float32), 8, 1)
        assert e.value.code == 1


def test_out_of_range_weight_is_rejected(oracle_mod):
    # t x_i >= 2^39 - 1 needs weight region 39
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.sketch([0, 1], np.array([1], np.uint32), np.array([2.0 ** 39], np.float32), 1, 1)
    assert e.value.code == 5


def test_sketch_is_seeded_and_keys_valid(oracle_mod):
    b = workloads.workload0(40)
    a1 = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1)
    a2 = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 2)
    assert (a1 != U64MAX).all()
    assert (a1 != a2).mean() > 0.99
    # rank codes are positive finite binary32 values below the final limit
    codes = (a1 >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.isfinite(codes).all() and (codes >= 0).all()
    # threads split the batch without changing results
    assert (oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1, threads=4) == a1).all()


def test_bbit_packing_matches_keys(oracle_mod):
    b = workloads.workload0(20)
    for bits in (1, 2, 4, 8, 16, 32):
        for k in (64, 100):
            words, keys = oracle_mod.sketch_bbit(b.indptr, b.indices, b.weights, k, bits, 4, keys=True)
            assert words.shape == (20, (k * bits + 63) // 64)
            full = oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 4)
            assert (keys == full).all()
            for s in range(3):
                for j in range(k):
                    beta = bf.mix64(int(keys[s, j]) ^ 0xA4093822299F31D0) & ((1 << bits) - 1)
                    wd, off = divmod(j * bits, 64)
                    assert (int(words[s, wd]) >> off) & ((1 << bits) - 1) == beta
                used = k * bits - 64 * (words.shape[1] - 1)
                if used < 64:
                    assert int(words[s, -1]) >> used == 0


def test_golden_tiny_sketches(oracle_mod):
    """Fixtures written by tests/golden/make_golden.py from the exact brute force."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_sketches.json")
    cases = json.load(open(path))["cases"]
    assert len(cases) >= 7
    for c in cases:
        w = np.array([float.fromhex(h) for h in c["weights_hex"]], dtype=np.float32)
        idx = np.array(c["indices"], dtype=np.uint32)
        assert oracle_mod.t_of_k(c["k"]) == c["t"]
        out = oracle_mod.sketch([0, len(idx)], idx, w, c["k"], c["seed"])[0]
        for j, h in enumerate(c["keys"]):
            if h is not None:
                assert int(out[j]) == int(h, 16), (c, j)


def test_zipf_generator_is_deterministic_and_distinct():
    b = workloads.zipf_batch(300, 5, 50, 1 << 16, 1.1, seed=7, threads=3)
    b2 = workloads.zipf_batch(300, 5, 50, 1 << 16, 1.1, seed=7, threads=1)
    assert (b.indices == b2.indices).all() and (b.weights == b2.weights).all()
    lens = np.diff(b.indptr)
    assert lens.min() >= 5 and lens.max() <= 50
    for s in range(300):
        row = b.indices[b.indptr[s]:b.indptr[s + 1]]
        assert len(set(row.tolist())) == len(row)
    assert (b.weights > 0.69).all() and (b.weights < 10 * np.log(1 + 1e6)).all()
