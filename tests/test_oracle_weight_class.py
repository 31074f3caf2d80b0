"""Pins of the oracle's weight-class normalisation for LSH (Section 3: split the data into classes
||x||_1 in [2^c, 2^(c+1)) and normalise each class to ||x||_1 in [1, 2)).  The normalisation is an
exact scaling of every weight by 2^scale:

- it equals hashing the weights multiplied by 2^scale in fp32 (exact for these powers of two);
- scale 0 is the plain method;
- the class is floor(log2 ||x||_1) of the exact sum of the positive finite weights, pinned at and
  next to powers of two (including a sum that binary64 addition rounds across a class edge), so
  normalised norms fall in [1, 2);
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


def edge_sets():
    """Sets whose class the definition fixes in closed form (Section 3's class edges
    ||x||_1 = 2^c), with the expected class of each."""
    f = np.float32
    below1 = float(np.nextafter(f(1), f(0)))                      # 1 - 2^-24
    fmax = float(np.finfo(np.float32).max)                        # (2 - 2^-23) 2^127
    rows = [
        ([2.0 ** -3] * 8, 0),                                     # exactly 1
        ([0.5, 0.25, 0.25], 0),
        ([2.0 ** 100, 2.0 ** 100], 101),
        ([2.0 ** -149], -149),                                    # the smallest subnormal
        ([2.0 ** -149] * 2, -148),
        ([2.0 ** -149] * 3, -148),
        ([1.0, below1], 0),                                       # 2 - 2^-24 (a binary32 sum rounds to 2)
        # exactly 2 - 2^-72: a binary64 sum rounds up to 2 (class 1); the exact class is 0
        ([1.0, below1, 2.0 ** -24 - 2.0 ** -48, 2.0 ** -48 - 2.0 ** -72], 0),
        ([1.0, below1, 2.0 ** -24], 1),                           # exactly 2
        ([fmax], 127),
        ([fmax, fmax], 128),                                      # beyond the binary32 range
        ([2.0 ** 127, 2.0 ** -149], 127),
        ([1.0, 2.0 ** -149], 0),
        ([float(np.nextafter(f(2), f(0)))], 0),
        ([2.0], 1),
        ([-1.0, 0.0, 0.5, float("inf"), float("nan")], -1),      # only positive finite weights count
        ([], 0),
        ([0.0, -2.0], 0),                                         # no positive weight
    ]
    for c in range(-149, 128, 7):
        rows.append(([2.0 ** c], c))
    return rows


def test_weight_class_edges(oracle_mod):
    rows = edge_sets()
    b = workloads.csr_of([(np.arange(len(w), dtype=np.uint32), np.array(w, dtype=np.float32)) for w, _ in rows])
    for w, _ in rows:                                             # every listed weight is a binary32 value
        assert np.array_equal(np.array(w, dtype=np.float32).astype(np.float64), np.array(w, dtype=np.float64),
                              equal_nan=True)
    got = oracle_mod.weight_class(b.indptr, b.weights)
    assert got.tolist() == [c for _, c in rows]
    # the crossing set really does cross under binary64 addition
    cross = np.array(rows[7][0], dtype=np.float64)
    assert cross.sum() == 2.0 and math.floor(math.log2(cross.sum())) == 1


def test_weight_class_bounds(oracle_mod):
    """On random sets over 16 decades: 2^c <= ||x||_1 < 2^(c+1) with the norm as an exact integer
    sum of the weights' significands on a common binary scale (2^-149), and the class does not
    depend on the order of the elements."""
    b = workloads.random_sets(300, 0, 40, 1 << 22, seed=13, scale_lo=1e-8, scale_hi=1e8)
    c = oracle_mod.weight_class(b.indptr, b.weights)
    bits = b.weights.view(np.uint32).astype(np.int64)
    for s in range(b.n_sets):
        n = 0
        for v in bits[b.indptr[s]:b.indptr[s + 1]].tolist():
            ex, fr = v >> 23, v & 0x7FFFFF
            if v >> 31 or ex == 255 or v == 0:
                continue
            n += (fr | (1 << 23) if ex else fr) << (max(ex, 1) - 1)       # x 2^149
        if n:
            assert 2 ** (int(c[s]) + 149) <= n < 2 ** (int(c[s]) + 150)
        else:
            assert c[s] == 0
    rng = np.random.default_rng(5)
    perm = b.rows(range(b.n_sets))
    for s in range(perm.n_sets):
        lo, hi = perm.indptr[s], perm.indptr[s + 1]
        perm.weights[lo:hi] = rng.permutation(perm.weights[lo:hi])
    assert np.array_equal(oracle_mod.weight_class(perm.indptr, perm.weights), c)


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
