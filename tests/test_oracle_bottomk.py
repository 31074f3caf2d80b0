"""Pins of the oracle's bottom-k weighted sketch (Section 3, "Bottom-k minhash"): t = k, phi raised
until DartHash returns at least k darts, the k smallest keys in increasing order.

- Exact: equal to the k smallest keys of a brute-force enumeration of the dart process over a
  box, whenever the box holds k darts below its rank bound (then no dart outside it can be
  smaller).
- Invariances: phi0, element order, zero weights; an empty set gives all ones.
- Statistics: the union estimator |S_k(x v y) n S_k(x) n S_k(y)| / k is Bin(k, J)/k for the
  weighted Jaccard J of Eq. 1 (every dart of the union process hits both sets with probability
  J, independently of its rank), checked in mean and dispersion over many pairs."""
import math

import numpy as np

import oracle.bruteforce as bf
import workloads

THREADS = 8
U64MAX = np.uint64(2 ** 64 - 1)


def _box(w, k, t, l1):
    y = max(float(x) * t for x in w)
    nu_box = 0
    while 2 ** (nu_box + 1) - 1 <= y:
        nu_box += 1
    R = 3.0 * k / (t * l1)           # rank bound holding about 3k darts
    rho_box = 0
    while 2 ** (rho_box + 1) - 1 < R:
        rho_box += 1
    return nu_box, rho_box


def test_bottomk_equals_bruteforce(oracle_mod):
    rng = np.random.default_rng(31)
    T = oracle_mod.poisson_thresholds()
    compared = 0
    for trial in range(40):
        k = int(rng.choice([1, 2, 3, 5, 8]))
        nnz = int(rng.integers(1, 5))
        idx = np.sort(rng.choice(5000, nnz, replace=False)).astype(np.uint32)
        w = (rng.random(nnz) * 10 ** rng.uniform(-1.0, 0.6) + 1e-6).astype(np.float32)
        l1 = float(w.astype(np.float64).sum())
        t = k
        nu_box, rho_box = _box(w, k, t, l1)
        if nnz * (2 ** (nu_box + 1)) * (2 ** (rho_box + 1)) > 60000:
            continue
        seed = int(rng.integers(0, 2 ** 62))
        o = oracle_mod.bottomk(np.array([0, nnz]), idx, w, k, seed)[0]
        b = bf.bottomk(idx, w, k, t, seed, nu_box, rho_box, T)
        if b is None:
            continue
        assert [int(v) for v in o] == b, (trial, k)
        compared += 1
    assert compared >= 20


def test_bottomk_sorted_and_invariant(oracle_mod):
    b = workloads.random_sets(120, 0, 60, 1 << 22, seed=41)
    k = 24
    ref = oracle_mod.bottomk(b.indptr, b.indices, b.weights, k, 5, threads=THREADS)
    nnz = np.diff(b.indptr)
    for s in range(b.n_sets):
        row = ref[s]
        if nnz[s] == 0:
            assert np.all(row == U64MAX)
        else:
            assert np.all(row[1:] > row[:-1])                # distinct darts, increasing keys
    for phi0 in (0.5, 2.0, 8.0):
        assert np.array_equal(oracle_mod.bottomk(b.indptr, b.indices, b.weights, k, 5, phi0=phi0,
                                                 threads=THREADS), ref)
    # element order and zero weights do not matter
    rng = np.random.default_rng(3)
    rows = []
    for s in range(b.n_sets):
        lo, hi = b.indptr[s], b.indptr[s + 1]
        p = rng.permutation(hi - lo)
        idx, w = b.indices[lo:hi][p], b.weights[lo:hi][p]
        rows.append((np.concatenate([idx, [7_000_000 + s]]).astype(np.uint32),
                     np.concatenate([w, [0.0]]).astype(np.float32)))
    c = workloads.csr_of(rows)
    assert np.array_equal(oracle_mod.bottomk(c.indptr, c.indices, c.weights, k, 5, threads=THREADS), ref)


def _union(ix, wx, iy, wy):
    d = {}
    for i, w in zip(ix, wx):
        d[int(i)] = max(d.get(int(i), 0.0), float(w))
    for i, w in zip(iy, wy):
        d[int(i)] = max(d.get(int(i), 0.0), float(w))
    keys = sorted(d)
    return np.array(keys, dtype=np.uint32), np.array([d[i] for i in keys], dtype=np.float32)


def test_bottomk_union_estimator_is_binomial(oracle_mod):
    rng = np.random.default_rng(77)
    k = 32
    pairs, jacc = [], []
    for target in (0.25, 0.5, 0.75):
        bpar = 2 * target / (1 + target)
        for _ in range(700):
            ix, wx, iy, wy = workloads.similar_pair(rng, 24, bpar)
            pairs.append((ix, wx, iy, wy))
            mx = dict(zip(ix.tolist(), wx.astype(np.float64).tolist()))
            my = dict(zip(iy.tolist(), wy.astype(np.float64).tolist()))
            keys = set(mx) | set(my)
            jacc.append(sum(min(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys)
                        / sum(max(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys))
    J = np.array(jacc)
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])
    us = workloads.csr_of([_union(*p) for p in pairs])
    seed = 123
    sx = oracle_mod.bottomk(xs.indptr, xs.indices, xs.weights, k, seed, threads=THREADS)
    sy = oracle_mod.bottomk(ys.indptr, ys.indices, ys.weights, k, seed, threads=THREADS)
    su = oracle_mod.bottomk(us.indptr, us.indices, us.weights, k, seed, threads=THREADS)
    c = np.array([len(set(su[i].tolist()) & set(sx[i].tolist()) & set(sy[i].tolist()))
                  for i in range(len(pairs))])
    mu, var = k * J.sum(), k * (J * (1 - J)).sum()
    assert abs(c.sum() - mu) / math.sqrt(var) < 3.5
    disp = (((c - k * J) ** 2) / (k * J * (1 - J))).sum()
    n = len(c)
    assert abs(disp - n) / math.sqrt(2.2 * n) < 4          # Bin(k, J) dispersion
