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


def test_topk_matches_a_plain_selection(oracle_mod):
    """compare_topk against a selection written out here: the topk rows by (count descending,
    row ascending), counts recounted slot by slot, padding past n_c."""
    rng = np.random.default_rng(21)
    k = 16
    a = rng.integers(0, 3, size=(7, k), dtype=np.uint64)
    c = rng.integers(0, 3, size=(23, k), dtype=np.uint64)
    for topk in (1, 5, 23, 30):
        rows, counts = oracle_mod.compare_topk(a, c, k, topk)
        for i in range(7):
            m = [sum(1 for q in range(k) if a[i, q] == c[j, q]) for j in range(23)]
            ranked = sorted(range(23), key=lambda j: (-m[j], j))[:topk]
            assert list(rows[i, :len(ranked)]) == ranked
            assert list(counts[i, :len(ranked)]) == [m[j] for j in ranked]
            assert np.all(rows[i, len(ranked):] == 0xFFFFFFFF) and np.all(counts[i, len(ranked):] == 0)
    rows, counts = oracle_mod.compare_topk(a, c[:0], k, 4)
    assert np.all(rows == 0xFFFFFFFF) and np.all(counts == 0)


def test_topk_finds_planted_copies(oracle_mod):
    """Through real sketches: a set's own sketch among others is its first neighbour with all k
    slots agreeing, and a near-duplicate (J = 0.9) outranks unrelated sets."""
    rng = np.random.default_rng(8)
    k, n = 128, 60
    base = workloads.random_sets(n, 20, 60, 1 << 20, seed=33)
    q_rows, near_rows = [], []
    for i in range(3):
        ix, wx, iy, wy = workloads.similar_pair(rng, 40, 2 * 0.9 / 1.9)     # J = 0.9
        q_rows.append((ix, wx))
        near_rows.append((iy, wy))
    qb = workloads.csr_of(q_rows)
    base_rows = [(base.indices[base.indptr[i]:base.indptr[i + 1]], base.weights[base.indptr[i]:base.indptr[i + 1]])
                 for i in range(n)]
    cb = workloads.csr_of(base_rows + near_rows + [q_rows[0]])
    qa = oracle_mod.sketch(qb.indptr, qb.indices, qb.weights, k, 4, threads=THREADS)
    ca = oracle_mod.sketch(cb.indptr, cb.indices, cb.weights, k, 4, threads=THREADS)
    rows, counts = oracle_mod.compare_topk(qa, ca, k, 3)
    assert rows[0, 0] == n + 3 and counts[0, 0] == k               # the planted copy of query 0
    for i in range(3):
        assert n + i in rows[i, :2]                                 # the J = 0.9 neighbour
