"""Pins of the oracle's weight-class normalisation for LSH (Section 3: split the data into classes
||x||_1 in [2^c, 2^(c+1)) and normalise each class to ||x||_1 in [1, 2)).  The normalisation is an
exact scaling of every weight by 2^scale:

- it equals hashing the weights multiplied by 2^scale in fp32 (exact for these powers of two);
- scale 0 is the plain method;
- the class is floor(log2 ||x||_1), so normalised norms fall in [1, 2);
- normalised pairs still collide with probability J^K per table (J is scale invariant)."""
import math

import numpy as np

import workloads

THREADS = 8


def test_scaling_equals_multiplied_weights(oracle_mod):
    b = workloads.random_sets(150, 1, 60, 1 << 22, seed=12, scale_lo=1e-2, scale_hi=1e2)
    rng = np.random.default_rng(4)
    scale = rng.integers(-6, 7, size=b.n_sets).astype(np.int32)
    got = oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 21, scale=scale, threads=THREADS)
    w2 = b.weights.copy()
    for s in range(b.n_sets):
        lo, hi = b.indptr[s], b.indptr[s + 1]
        w2[lo:hi] = (b.weights[lo:hi].astype(np.float64) * 2.0 ** int(scale[s])).astype(np.float32)
        assert np.array_equal(w2[lo:hi].astype(np.float64), b.weights[lo:hi].astype(np.float64) * 2.0 ** int(scale[s]))
    ref = oracle_mod.lsh(b.indptr, b.indices, w2, 32, 4, 21, threads=THREADS)
    assert np.array_equal(got, ref)
    plain = oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 21, threads=THREADS)
    assert np.array_equal(oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 21, threads=THREADS,
                                         scale=np.zeros(b.n_sets, np.int32)), plain)


def test_weight_class_bounds(oracle_mod):
    b = workloads.random_sets(300, 0, 40, 1 << 22, seed=13, scale_lo=1e-6, scale_hi=1e6)
    c = oracle_mod.weight_class(b.indptr, b.weights)
    for s in range(b.n_sets):
        l1 = float(b.weights[b.indptr[s]:b.indptr[s + 1]].astype(np.float64).sum())
        if l1 > 0:
            assert 1.0 <= l1 * 2.0 ** -int(c[s]) < 2.0
        else:
            assert c[s] == 0


def test_normalised_pairs_collide_at_j_to_the_k(oracle_mod):
    """Pairs of the paper's recipe scaled by a common random factor, hashed with their class's
    normalisation: per-table collisions at J^K."""
    rng = np.random.default_rng(19)
    L, K, target = 32, 2, 0.6
    bpar = 2 * target / (1 + target)
    xs, ys = [], []
    for _ in range(1500):
        ix, wx, iy, wy = workloads.similar_pair(rng, 24, bpar)
        f = np.float32(2.0 ** rng.uniform(-8, 8))
        xs.append((ix, (wx * f).astype(np.float32)))
        ys.append((iy, (wy * f).astype(np.float32)))
    bx, by = workloads.csr_of(xs), workloads.csr_of(ys)
    cx = oracle_mod.weight_class(bx.indptr, bx.weights)
    # both members of a pair go through the same class (the query side probes its partner's)
    vx = oracle_mod.lsh(bx.indptr, bx.indices, bx.weights, L, K, 5, scale=-cx, threads=THREADS)
    vy = oracle_mod.lsh(by.indptr, by.indices, by.weights, L, K, 5, scale=-cx, threads=THREADS)
    J = []
    for (ix, wx), (iy, wy) in zip(xs, ys):
        mx = dict(zip(ix.tolist(), wx.astype(np.float64).tolist()))
        my = dict(zip(iy.tolist(), wy.astype(np.float64).tolist()))
        keys = set(mx) | set(my)
        J.append(sum(min(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys)
                 / sum(max(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys))
    p = np.array(J) ** K
    hits = (vx == vy).sum()
    mu, var = L * p.sum(), L * (p * (1 - p)).sum()
    assert abs(hits - mu) / math.sqrt(var) < 4
