"""Seeded synthetic weighted-set generators shared by the tests, the bench and the oracle legs.

This module holds no part of the method's arithmetic (no hashing, no dart logic): it only
draws CSR batches of weighted sets with numpy's PCG64 generator, following the recipes
below.  Data seed = 1000 + workload number; every call with the same arguments returns the
same arrays.

  W0  1,000 sets, universe d = 100,000, 64 distinct uniform indices per set (sorted),
      weights Uniform(0, 1] fp32 (drawn as 1 - u).                         k = 64
  W1  1,000,000 sets, d = 2^20, 256 distinct uniform indices, weights Exponential(1) fp32.
                                                                   k = 256 and 1-bit
  W2  200,000 sets, d = 2^24, nnz = round(exp(ln 100 + 1.5 z)) clipped to [1, 100,000],
      weights lognormal(0, 1) rescaled per set so ||x||_1 = 10^U(-3, 3).          k = 1024
  W3  1,000,000 tf-idf-like sets over d = 2^20: nnz ~ Uniform{200..2000}; tokens drawn from
      Zipf(1.1) over the universe until nnz distinct elements appear; weight = log(1 + count)
      x Uniform(1, 10) (token sampling in zipf_gen.c).                         L = 64, K = 8
  W4  request stream: Poisson arrivals at 50,000/s; nnz = min(100,000, floor(Pareto(1.2)))
      with x_m = 1; d = 2^24; weights Uniform(0, 5]; k uniform over {64, 256, 1024}.

Plus the pair recipe of the paper's Section 4 ("Synthetic data"): y_i = b x_i on supp(x)
and y_j = 1 - b on one fresh element j, with ||x||_1 = 1, so J(x, y) = b / (2 - b).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))


@dataclass
class Batch:
    indptr: np.ndarray      # int64[n + 1]
    indices: np.ndarray     # uint32[nnz]
    weights: np.ndarray     # float32[nnz]
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def n_sets(self) -> int:
        return len(self.indptr) - 1

    @property
    def nnz(self) -> int:
        return int(self.indptr[-1])

    def rows(self, sel):
        """Sub-batch of the given row numbers (copied, re-based CSR)."""
        sel = np.asarray(sel, dtype=np.int64)
        lens = self.indptr[sel + 1] - self.indptr[sel]
        ip = np.zeros(len(sel) + 1, dtype=np.int64)
        np.cumsum(lens, out=ip[1:])
        take = np.concatenate([np.arange(self.indptr[s], self.indptr[s + 1]) for s in sel]) \
            if len(sel) else np.zeros(0, dtype=np.int64)
        return Batch(ip, self.indices[take].copy(), self.weights[take].copy(), self.name,
                     dict(self.params, rows=len(sel)))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def distinct_sorted_rows(rng, n: int, m: int, d: int) -> np.ndarray:
    """n rows of m distinct indices uniform on [0, d), each row sorted ascending."""
    out = np.sort(rng.integers(0, d, size=(n, m), dtype=np.int64), axis=1)
    while True:
        bad = np.nonzero((np.diff(out, axis=1) == 0).any(axis=1))[0] if m > 1 else np.zeros(0, int)
        if len(bad) == 0:
            return out.astype(np.uint32)
        out[bad] = np.sort(rng.integers(0, d, size=(len(bad), m), dtype=np.int64), axis=1)


def fixed_nnz_batch(n: int, nnz: int, d: int, weight: str, seed: int, name: str = "") -> Batch:
    rng = _rng(seed)
    idx = distinct_sorted_rows(rng, n, nnz, d).reshape(-1)
    if weight == "uniform01":
        w = (1.0 - rng.random(n * nnz, dtype=np.float32)).astype(np.float32)
    elif weight == "exp1":
        w = rng.standard_exponential(n * nnz, dtype=np.float32)
    else:
        raise ValueError(weight)
    ip = np.arange(0, (n + 1) * nnz, nnz, dtype=np.int64)
    return Batch(ip, idx, w, name, dict(n=n, nnz=nnz, d=d, weight=weight, seed=seed))


def workload0(n: int = 1000) -> Batch:
    """W0: 1,000 sets x 64 distinct indices over d = 100,000, weights U(0, 1]."""
    return fixed_nnz_batch(n, 64, 100_000, "uniform01", 1000, "W0")


def workload1(n: int = 1_000_000, shard: int = 0) -> Batch:
    """W1: 1,000,000 sets x 256 distinct indices over d = 2^20, weights Exp(1).  shard > 0 draws
    another batch of the same distribution (data seed 1001 + 1000 shard), one per rank."""
    return fixed_nnz_batch(n, 256, 1 << 20, "exp1", 1001 + 1000 * shard, "W1")


def _ragged_distinct(rng, lens: np.ndarray, d: int) -> np.ndarray:
    """Concatenated rows of distinct uniform indices on [0, d) with the given lengths,
    each row sorted."""
    n = len(lens)
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    row = np.repeat(np.arange(n, dtype=np.int64), lens)
    vals = rng.integers(0, d, size=int(ip[-1]), dtype=np.int64)
    while True:
        key = row * d + vals
        order = np.argsort(key, kind="stable")
        key = key[order]
        vals = vals[order]
        dup = np.zeros(len(key), dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        if not dup.any():
            return vals.astype(np.uint32)
        vals[dup] = rng.integers(0, d, size=int(dup.sum()), dtype=np.int64)


def workload2(n: int = 200_000, shard: int = 0) -> Batch:
    """W2: heavy-tailed nnz (log-normal, median 100, sigma 1.5, clipped to [1, 1e5]) over
    d = 2^24; weights lognormal(0, 1) rescaled so ||x||_1 is log-uniform on [1e-3, 1e3].
    shard > 0 draws another batch of the same distribution (data seed 1002 + 1000 shard)."""
    rng = _rng(1002 + 1000 * shard)
    lens = np.clip(np.rint(np.exp(np.log(100.0) + 1.5 * rng.standard_normal(n))), 1, 100_000)
    lens = lens.astype(np.int64)
    idx = _ragged_distinct(rng, lens, 1 << 24)
    z = rng.lognormal(0.0, 1.0, size=int(lens.sum()))
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    target = 10.0 ** rng.uniform(-3.0, 3.0, size=n)
    sums = np.add.reduceat(z, ip[:-1])
    w = (z * np.repeat(target / sums, lens)).astype(np.float32)
    return Batch(ip, idx, w, "W2", dict(n=n, d=1 << 24, seed=1002))


_gen_lock = threading.Lock()
_gen_lib = None
_alias_cache = {}


def _zipf_lib():
    """The tf-idf token sampler (zipf_gen.c), compiled in-tree on first use."""
    global _gen_lib
    with _gen_lock:
        if _gen_lib is None:
            src = os.path.join(_HERE, "zipf_gen.c")
            out = os.path.join(_HERE, "_build", "libzipfgen.so")
            os.makedirs(os.path.dirname(out), exist_ok=True)
            if not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
                tmp = out + f".tmp{os.getpid()}"
                subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
                os.replace(tmp, out)
            lib = ctypes.CDLL(out)
            P = ctypes.c_void_p
            lib.zipf_alias.argtypes = [ctypes.c_int64, ctypes.c_double, P, P]
            lib.zipf_sets.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_int64, P, P, P, P]
            _gen_lib = lib
        return _gen_lib


def _zipf_tables(d: int, s: float):
    key = (d, s)
    if key not in _alias_cache:
        prob = np.empty(d, dtype=np.float64)
        alias = np.empty(d, dtype=np.int32)
        assert _zipf_lib().zipf_alias(d, s, prob.ctypes.data, alias.ctypes.data) == 0
        _alias_cache[key] = (prob, alias)
    return _alias_cache[key]


def zipf_batch(n: int, nnz_lo: int, nnz_hi: int, d: int, s: float, seed: int, threads: int | None = None,
               name: str = "zipf") -> Batch:
    """Sets of nnz ~ U{nnz_lo..nnz_hi} distinct elements drawn from Zipf(s) token streams,
    weight = log(1 + count) x U(1, 10)."""
    rng = _rng(seed)
    lens = rng.integers(nnz_lo, nnz_hi + 1, size=n).astype(np.int64)
    seeds = rng.integers(1, 2 ** 63, size=(n, 4), dtype=np.int64).view(np.uint64)
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    idx = np.empty(int(ip[-1]), dtype=np.uint32)
    w = np.empty(int(ip[-1]), dtype=np.float32)
    prob, alias = _zipf_tables(d, s)
    lib = _zipf_lib()
    threads = threads or os.cpu_count() or 1
    bounds = np.linspace(0, n, 4 * threads + 1).astype(np.int64)

    def run(c):
        a, b = int(bounds[c]), int(bounds[c + 1])
        if b > a:
            return lib.zipf_sets(a, b, ip.ctypes.data, seeds.ctypes.data, d, prob.ctypes.data, alias.ctypes.data,
                                 idx.ctypes.data, w.ctypes.data)
        return 0

    with ThreadPoolExecutor(threads) as ex:
        assert all(rc == 0 for rc in ex.map(run, range(len(bounds) - 1)))
    return Batch(ip, idx, w, name, dict(n=n, d=d, zipf=s, seed=seed))


def workload3(n: int = 1_000_000, threads: int | None = None, shard: int = 0) -> Batch:
    """W3: tf-idf-like sets for (L, K) = (64, 8) LSH (see the module docstring).  shard > 0 draws
    another batch of the same distribution (data seed 1003 + 1000 shard)."""
    return zipf_batch(n, 200, 2000, 1 << 20, 1.1, 1003 + 1000 * shard, threads, "W3")


def workload4_requests(rate: float = 50_000.0, seconds: float = 60.0, max_requests: int | None = None):
    """W4 request stream: (arrival times [s], Batch of one set per request, k per request)."""
    rng = _rng(1004)
    n = int(rng.poisson(rate * seconds))
    if max_requests is not None:
        n = min(n, max_requests)
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps)
    lens = np.minimum(100_000, np.floor(rng.pareto(1.2, size=n) + 1.0)).astype(np.int64)
    idx = _ragged_distinct(rng, lens, 1 << 24)
    w = (5.0 * (1.0 - rng.random(int(lens.sum())))).astype(np.float32)
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    ks = rng.choice(np.array([64, 256, 1024], dtype=np.int32), size=n)
    return arrivals, Batch(ip, idx, w, "W4", dict(n=n, rate=rate, seed=1004)), ks


def random_sets(n: int, nnz_lo: int, nnz_hi: int, d: int, seed: int, scale_lo=1e-3, scale_hi=1e3,
                name="random") -> Batch:
    """Test batch with ragged nnz in [nnz_lo, nnz_hi] and ||x||_1 log-uniform on
    [scale_lo, scale_hi] (weights lognormal before scaling)."""
    rng = _rng(seed)
    lens = rng.integers(nnz_lo, nnz_hi + 1, size=n).astype(np.int64)
    idx = _ragged_distinct(rng, lens, d)
    z = rng.lognormal(0.0, 1.0, size=int(lens.sum()))
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    if n and lens.min() > 0:
        target = np.exp(rng.uniform(np.log(scale_lo), np.log(scale_hi), size=n))
        sums = np.add.reduceat(z, ip[:-1])
        z = z * np.repeat(target / sums, lens)
    return Batch(ip, idx, z.astype(np.float32), name, dict(n=n, seed=seed))


def simplex_set(rng, nnz: int, l1: float = 1.0, d: int = 1 << 32):
    """Section 4's synthetic set: a uniform point of the probability simplex (normalised
    Exp(1) draws) scaled to ||x||_1 = l1, on nnz distinct random elements."""
    idx = np.sort(rng.choice(d, size=nnz, replace=False)).astype(np.uint32) if d <= 1 << 24 else \
        distinct_sorted_rows(rng, 1, nnz, d)[0]
    e = rng.standard_exponential(nnz)
    return idx, (l1 * e / e.sum()).astype(np.float32)


def similar_pair(rng, nnz: int, b: float, d: int = 1 << 30):
    """Section 4's pair: x on the simplex (||x||_1 = 1), y_i = b x_i, plus y_j = 1 - b on an
    element j outside supp(x).  Returns (idx_x, w_x, idx_y, w_y)."""
    idx = distinct_sorted_rows(rng, 1, nnz + 1, d)[0]
    perm = rng.permutation(nnz + 1)
    ix, extra = np.sort(idx[perm[:nnz]]), idx[perm[nnz]]
    e = rng.standard_exponential(nnz)
    wx = (e / e.sum()).astype(np.float32)
    wy = (np.float32(b) * wx).astype(np.float32)
    iy = np.concatenate([ix, [extra]]).astype(np.uint32)
    wyy = np.concatenate([wy, [np.float32(1.0 - b)]]).astype(np.float32)
    o = np.argsort(iy)
    return ix, wx, iy[o], wyy[o]


def csr_of(rows) -> Batch:
    """CSR Batch from a list of (indices, weights) rows."""
    lens = np.array([len(r[0]) for r in rows], dtype=np.int64)
    ip = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    idx = np.concatenate([np.asarray(r[0], dtype=np.uint32) for r in rows]) if rows else np.zeros(0, np.uint32)
    w = np.concatenate([np.asarray(r[1], dtype=np.float32) for r in rows]) if rows else np.zeros(0, np.float32)
    return Batch(ip, idx.astype(np.uint32), w.astype(np.float32), "rows")


# ------------------------------------------------------------------------------------------
# 64-bit ids and binary64 weights (Section 4, "Synthetic data", as the paper states it; Table 1)
# ------------------------------------------------------------------------------------------
@dataclass
class WideBatch:
    indptr: np.ndarray      # int64[n + 1]
    indices: np.ndarray     # uint64[nnz]
    weights: np.ndarray     # float64[nnz]
    name: str = ""

    @property
    def n_sets(self) -> int:
        return len(self.indptr) - 1


def wide_ids(rng, n: int) -> np.ndarray:
    """n distinct uniform 64-bit element ids (sorted)."""
    while True:
        ids = np.unique(rng.integers(0, 2 ** 64, size=n, dtype=np.uint64, endpoint=False))
        if len(ids) == n:
            return ids


def wide_set(rng, nnz: int, l1: float):
    """A uniform point of the probability simplex (normalised Exp(1) draws) scaled to
    ||x||_1 = l1 (an exact power-of-two scaling for l1 = 2^e), on nnz distinct random 64-bit ids."""
    e = rng.standard_exponential(nnz)
    return wide_ids(rng, nnz), (e / e.sum()) * np.float64(l1)


def wide_pair(rng, nnz: int, b: float, l1: float):
    """The pair recipe at norm l1: x = wide_set, y_i = b x_i on supp(x) and y_j = (1 - b) l1 on
    one fresh id j, so J(x, y) = b / (2 - b) and ||y||_1 = ||x||_1.  Returns (ix, wx, iy, wy)."""
    ids = wide_ids(rng, nnz + 1)
    perm = rng.permutation(nnz + 1)
    ix, extra = np.sort(ids[perm[:nnz]]), ids[perm[nnz]]
    e = rng.standard_exponential(nnz)
    wx = (e / e.sum()) * np.float64(l1)
    iy = np.concatenate([ix, [extra]])
    wy = np.concatenate([b * wx, [(1.0 - b) * np.float64(l1)]])
    o = np.argsort(iy)
    return ix, wx, iy[o], wy[o]


def wide_csr(rows, name: str = "rows") -> WideBatch:
    lens = np.array([len(r[0]) for r in rows], dtype=np.int64)
    ip = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    idx = np.concatenate([np.asarray(r[0], dtype=np.uint64) for r in rows]) if rows else np.zeros(0, np.uint64)
    w = np.concatenate([np.asarray(r[1], dtype=np.float64) for r in rows]) if rows else np.zeros(0, np.float64)
    return WideBatch(ip, idx, w, name)


def table1_batch(n: int, nnz: int, l1: float, seed: int) -> WideBatch:
    """Table 1's rows: n sets of nnz elements at ||x||_1 = l1 (Section 4's recipe)."""
    rng = _rng(seed)
    return wide_csr([wide_set(rng, nnz, l1) for _ in range(n)], f"table1 nnz={nnz} l1={l1!r}")
