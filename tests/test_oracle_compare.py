"""Pins of the oracle's sketch comparison (Section 1.1): the counts equal a slot-by-slot loop
written independently here, and through real sketches they follow Eq. 1 (E[m] = k J for
minhash keys) and the b-bit collision law E[m] = k (J + (1 - J) 2^-b)."""
import math

import numpy as np
import pytest

import workloads

THREADS = 8


def test_compare_matches_a_plain_loop(oracle_mod):
    rng = np.random.default_rng(5)
    k = 37
    a = rng.integers(0, 4, size=(6, k), dtype=np.uint64)
    c = rng.integers(0, 4, size=(6, k), dtype=np.uint64)
    got = oracle_mod.compare(a, c, k)
    for i in range(6):
        assert got[i] == sum(1 for j in range(k) if a[i, j] == c[i, j])
    cross = oracle_mod.compare(a, c, k, mode="cross")
    for i in range(6):
        for j in range(6):
            assert cross[i, j] == sum(1 for q in range(k) if a[i, q] == c[j, q])
    for bits in (1, 2, 4, 8, 16, 32):
        W = (k * bits + 63) // 64
        wa = rng.integers(0, 2 ** 63, size=(5, W), dtype=np.uint64)
        wc = wa.copy()
        wc[:, 0] ^= np.uint64(1) << np.uint64(rng.integers(0, 64))
        used = k * bits - 64 * (W - 1)
        if used < 64:                                   # unused high bits of the last word are zero
            wa[:, -1] &= np.uint64((1 << used) - 1)
            wc[:, -1] &= np.uint64((1 << used) - 1)
        got = oracle_mod.compare(wa, wc, k, bits=bits)
        for i in range(5):
            ref = 0
            for j in range(k):
                pa = (int(wa[i, (j * bits) // 64]) >> ((j * bits) % 64)) & ((1 << bits) - 1)
                pc = (int(wc[i, (j * bits) // 64]) >> ((j * bits) % 64)) & ((1 << bits) - 1)
                ref += pa == pc
            assert got[i] == ref


@pytest.mark.parametrize("bits", [0, 1, 4])
def test_compare_follows_the_collision_laws(oracle_mod, bits):
    rng = np.random.default_rng(100 + bits)
    target, k = 0.5, 64
    bpar = 2 * target / (1 + target)
    pairs = [workloads.similar_pair(rng, 32, bpar) for _ in range(3000)]
    J = []
    for ix, wx, iy, wy in pairs:
        mx = dict(zip(ix.tolist(), wx.astype(np.float64).tolist()))
        my = dict(zip(iy.tolist(), wy.astype(np.float64).tolist()))
        keys = set(mx) | set(my)
        J.append(sum(min(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys)
                 / sum(max(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys))
    J = np.array(J)
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])
    if bits == 0:
        a = oracle_mod.sketch(xs.indptr, xs.indices, xs.weights, k, 9, threads=THREADS)
        c = oracle_mod.sketch(ys.indptr, ys.indices, ys.weights, k, 9, threads=THREADS)
    else:
        a = oracle_mod.sketch_bbit(xs.indptr, xs.indices, xs.weights, k, bits, 9, threads=THREADS)
        c = oracle_mod.sketch_bbit(ys.indptr, ys.indices, ys.weights, k, bits, 9, threads=THREADS)
    m = oracle_mod.compare(a, c, k, bits=bits).astype(np.float64)
    p = J + (1 - J) * (2.0 ** -bits if bits else 0.0)
    assert abs(m.sum() - k * p.sum()) / math.sqrt(k * (p * (1 - p)).sum()) < 4


def test_estimator_is_unbiased_and_fixes_its_end_points(oracle_mod):
    """Section 1.1: with m ~ Bin(k, J + (1 - J) 2^-b) agreeing b-bit fields (p = J for keys), the
    estimate has expectation exactly J (summed over the binomial pmf in rationals); all slots
    agreeing gives 1, and the chance level k 2^-b gives 0."""
    from fractions import Fraction
    from math import comb
    k = 64
    for bits in (0, 1, 2, 4, 8):
        m = np.arange(k + 1, dtype=np.uint32)
        est = oracle_mod.estimate_jaccard(m, k, bits=bits)
        assert est[k] == 1.0
        if bits and (k >> bits) << bits == k:
            assert est[k >> bits] == 0.0
        for J in (Fraction(1, 5), Fraction(1, 2), Fraction(7, 8)):
            p = J if bits == 0 else J + (1 - J) / 2 ** bits
            mean = sum(comb(k, i) * p ** i * (1 - p) ** (k - i) * Fraction(float(est[i])) for i in range(k + 1))
            assert abs(float(mean - J)) < 1e-12, (bits, J)
