"""Pins of the oracle's LSH-table query (Sections 1.2 and 3): on a hand-made instance the
candidates are the points sharing a value with the query in some table; on LSH values of real
sets, a point similar to the query is found with probability 1 - (1 - J^K)^L."""
import math

import numpy as np

import workloads

THREADS = 8


def test_index_query_small_instance(oracle_mod):
    values = np.array([[1, 2], [1, 3], [4, 2], [5, 6]], dtype=np.uint32)
    ids = np.array([10, 11, 12, 13], dtype=np.int64)
    queries = np.array([[1, 2], [5, 9], [7, 7], [4, 3]], dtype=np.uint32)
    counts, out = oracle_mod.lsh_index_query(values, ids, queries, 2)
    assert counts.tolist() == [3, 1, 0, 2]
    assert out.tolist() == [[10, 11], [13, -1], [-1, -1], [11, 12]]


def test_index_recall_follows_the_lsh_law(oracle_mod):
    rng = np.random.default_rng(12)
    L, K, target = 16, 3, 0.7
    bpar = 2 * target / (1 + target)
    pairs = [workloads.similar_pair(rng, 24, bpar) for _ in range(800)]
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])
    vx = oracle_mod.lsh(xs.indptr, xs.indices, xs.weights, L, K, 3, threads=THREADS)
    vy = oracle_mod.lsh(ys.indptr, ys.indices, ys.weights, L, K, 3, threads=THREADS)
    counts, out = oracle_mod.lsh_index_query(vx, np.arange(len(pairs)), vy, 64)
    found = np.array([i in out[i] for i in range(len(pairs))])
    J = []
    for ix, wx, iy, wy in pairs:
        mx = dict(zip(ix.tolist(), wx.astype(np.float64).tolist()))
        my = dict(zip(iy.tolist(), wy.astype(np.float64).tolist()))
        keys = set(mx) | set(my)
        J.append(sum(min(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys)
                 / sum(max(mx.get(i, 0.0), my.get(i, 0.0)) for i in keys))
    p = 1 - (1 - np.array(J) ** K) ** L
    assert abs(found.sum() - p.sum()) / math.sqrt((p * (1 - p)).sum()) < 4
    assert np.all(counts <= len(pairs))
