"""DartMinHash ORACLE -- test infrastructure only.

A plain CPU statement of the method of T. Christiani, "DartMinHash: Fast Sketching for
Weighted Sets" (arXiv 2005.11547).  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` leg / ``--impl reference`` arm may import this package.
It shares no code, header, table or constant generator with the CUDA library in
``paper_2005_11547_gb300``, and neither side imports the other.

Contents
  * ``t_of_k`` -- t = ceil(k ln k) + k (Theorem 1), from a 60-digit decimal logarithm.
  * ``poisson_thresholds`` -- the inversion table for X ~ Poi(1) (Algorithm 1, "X ~ Poi(1)";
    Section 4, "Implementation": a precomputed Poisson CDF table), exact to the last bit.
  * ``sketch`` / ``sketch_bbit`` / ``lsh`` / ``darthash`` -- thin ctypes calls into
    ``dm_oracle.c`` (Algorithm 1, Theorem 1, b-bit minhash, (L, K) LSH).
  * ``bruteforce`` -- an independent exact-Fraction enumeration of the hashed dart process
    over a bounding box, used to pin the C code.
  * ``wide`` -- the wide-range variant (binary64 weights, 64-bit element ids, the norms of
    Table 1) in pure Python integers, with its own box brute force.

Parity of the hash bits themselves is unpinned by the paper (it prints no hash values and
uses random tabulation tables); they are pinned only by the statistical tests in
``tests/test_oracle_stats.py`` and by the brute force.
"""
from __future__ import annotations

import ctypes
import decimal
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libdmoracle.so")

ERRORS = {0: "ok", 1: "invalid argument", 2: "out of memory", 5: "out of supported range",
          6: "phi limit reached"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, '?')}")
        self.code = code


# ------------------------------------------------------------------------------------------
# build / load
# ------------------------------------------------------------------------------------------
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile dm_oracle.c (plain C, no contraction of a*b+c, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64, dbl, flt = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_float)
        lib.dmo_sketch.argtypes = [P, P, P, i64, i32, u64, i64, P, dbl, i32, P, P]
        lib.dmo_sketch.restype = ctypes.c_int
        lib.dmo_sketch_bbit.argtypes = [P, P, P, i64, i32, i32, u64, i64, P, P, P]
        lib.dmo_sketch_bbit.restype = ctypes.c_int
        lib.dmo_lsh.argtypes = [P, P, P, i64, i32, i32, u64, P, dbl, P, P]
        lib.dmo_lsh.restype = ctypes.c_int
        lib.dmo_lsh_scaled.argtypes = [P, P, P, i64, i32, i32, u64, P, dbl, P, P, P]
        lib.dmo_lsh_scaled.restype = ctypes.c_int
        lib.dmo_bottomk.argtypes = [P, P, P, i64, i32, u64, P, dbl, P, P]
        lib.dmo_bottomk.restype = ctypes.c_int
        lib.dmo_darthash.argtypes = [P, P, i64, i64, u64, P, flt, P, i64, P]
        lib.dmo_darthash.restype = ctypes.c_int64
        lib.dmo_dart_record_size.restype = ctypes.c_int64
        lib.dmo_mix64.argtypes = [u64]
        lib.dmo_mix64.restype = u64
        assert lib.dmo_dart_record_size() == DART_DTYPE.itemsize
        _lib = lib
        return lib


# ------------------------------------------------------------------------------------------
# exact constants
# ------------------------------------------------------------------------------------------
def t_of_k(k: int) -> int:
    """t = ceil(k ln k) + k (Theorem 1's proof).  k ln k is irrational for k >= 2, so a
    60-digit logarithm decides the ceiling; the margin is asserted."""
    if k < 1:
        raise ValueError("k >= 1")
    if k == 1:
        return 1
    with decimal.localcontext() as c:
        c.prec = 60
        v = decimal.Decimal(k) * decimal.Decimal(k).ln()
        f = int(v.to_integral_value(rounding=decimal.ROUND_CEILING))
        assert f - v > decimal.Decimal("1e-40") and v - (f - 1) > decimal.Decimal("1e-40")
    return f + k


def _einv_bounds(terms: int = 60):
    """Rational lower/upper bounds on e^{-1} from its alternating series."""
    s, term = Fraction(0), Fraction(1)
    for l in range(terms):
        s += term if l % 2 == 0 else -term
        term /= (l + 1)
    return s - term, s + term


def poisson_thresholds() -> np.ndarray:
    """T[n] = ceil(2^32 * P(Poi(1) <= n)) for n = 0..11 (T[12] would be 2^32).

    With u uniform on [0, 2^32), X = #{n : u >= T[n]} has P(X = n) = (T[n] - T[n-1]) / 2^32,
    i.e. the Poisson(1) pmf to within 2^-32, and X <= 12."""
    lo, hi = _einv_bounds()
    out, cum, fact = [], Fraction(0), Fraction(1)
    for n in range(12):
        if n:
            fact /= n
        cum += fact
        a, b = lo * cum * 2 ** 32, hi * cum * 2 ** 32
        ca, cb = -((-a.numerator) // a.denominator), -((-b.numerator) // b.denominator)
        assert ca == cb, "bounds too loose"
        out.append(ca)
    assert out[-1] < 2 ** 32
    return np.array(out, dtype=np.uint32)


_T = None


def _table():
    global _T
    if _T is None:
        _T = np.ascontiguousarray(poisson_thresholds())
    return _T


# ------------------------------------------------------------------------------------------
# calls
# ------------------------------------------------------------------------------------------
def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _csr(indptr, indices, weights):
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.uint32)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    assert indptr.ndim == 1 and indptr[0] == 0 and indptr[-1] <= len(indices) == len(weights)
    return indptr, indices, weights


def _chunks(n, threads):
    threads = max(1, min(threads, n))
    b = np.linspace(0, n, threads + 1).astype(np.int64)
    return [(int(b[i]), int(b[i + 1])) for i in range(threads) if b[i + 1] > b[i]]


def _run_chunked(n, threads, fn):
    ch = _chunks(n, threads)
    if len(ch) <= 1:
        rcs = [fn(0, n)] if n else [0]
    else:
        with ThreadPoolExecutor(len(ch)) as ex:
            rcs = list(ex.map(lambda c: fn(*c), ch))
    rc = next((r for r in rcs if r), 0)
    if rc:
        raise OracleError(rc)


def sketch(indptr, indices, weights, k: int, seed: int, *, phi0: float = 1.0,
           schedule: str = "double", threads: int = 1, work: bool = False):
    """k minhash keys per row (uint64[n, k]); Theorem 1 with Algorithm 1 as inner step.
    ``schedule`` 'double' (phi <- 2 phi) or 'step' (phi <- phi + 1, Theorem 1's literal loop).
    With ``work=True`` also returns int64[n, 4]: areas, darts, kept darts, passes."""
    lib = _load()
    indptr, indices, weights = _csr(indptr, indices, weights)
    n = len(indptr) - 1
    out = np.empty((n, k), dtype=np.uint64)
    wk = np.zeros((n, 4), dtype=np.int64)
    t, T = t_of_k(k), _table()
    sch = {"double": 0, "step": 1}[schedule]

    def fn(a, b):
        ip = indptr[a:b + 1]
        return lib.dmo_sketch(_ptr(ip), _ptr(indices), _ptr(weights), b - a, k, seed & (2**64 - 1),
                              t, _ptr(T), float(phi0), sch,
                              ctypes.c_void_p(out.ctypes.data + a * k * 8),
                              ctypes.c_void_p(wk.ctypes.data + a * 32))

    _run_chunked(n, threads, fn)
    return (out, wk) if work else out


def sketch_bbit(indptr, indices, weights, k: int, b: int, seed: int, *, threads: int = 1,
                keys: bool = False):
    """b-bit packed sketches: uint64[n, ceil(k b / 64)] (and the uint64 keys if asked)."""
    lib = _load()
    indptr, indices, weights = _csr(indptr, indices, weights)
    n = len(indptr) - 1
    words = (k * b + 63) // 64
    out = np.empty((n, words), dtype=np.uint64)
    kout = np.empty((n, k), dtype=np.uint64) if keys else None
    t, T = t_of_k(k), _table()

    def fn(a, e):
        ip = indptr[a:e + 1]
        return lib.dmo_sketch_bbit(_ptr(ip), _ptr(indices), _ptr(weights), e - a, k, b,
                                   seed & (2**64 - 1), t, _ptr(T),
                                   ctypes.c_void_p(out.ctypes.data + a * words * 8),
                                   ctypes.c_void_p(kout.ctypes.data + a * k * 8) if keys else None)

    _run_chunked(n, threads, fn)
    return (out, kout) if keys else out


def lsh(indptr, indices, weights, L: int, K: int, seed: int, *, phi0: float = 1.0,
        threads: int = 1, work: bool = False, scale=None):
    """(L, K) LSH values uint32[n, L] (t = L K, L buckets, hash of the sorted bottom-K keys).
    scale (int32[n], optional): set s's weights count as x_i 2^scale[s] (Section 3's weight-class
    normalisation, exact)."""
    lib = _load()
    indptr, indices, weights = _csr(indptr, indices, weights)
    n = len(indptr) - 1
    out = np.empty((n, L), dtype=np.uint32)
    wk = np.zeros((n, 4), dtype=np.int64)
    T = _table()
    sc = None if scale is None else np.ascontiguousarray(scale, dtype=np.int32)

    def fn(a, b):
        ip = indptr[a:b + 1]
        return lib.dmo_lsh_scaled(_ptr(ip), _ptr(indices), _ptr(weights), b - a, L, K, seed & (2**64 - 1),
                                  _ptr(T), float(phi0), None if sc is None else ctypes.c_void_p(sc.ctypes.data + a * 4),
                                  ctypes.c_void_p(out.ctypes.data + a * L * 4),
                                  ctypes.c_void_p(wk.ctypes.data + a * 32))

    _run_chunked(n, threads, fn)
    return (out, wk) if work else out


def lsh_index_query(values, ids, queries, max_candidates: int):
    """Approximate near neighbor candidates of the (L, K) LSH tables (Section 1.2, "Fast similarity
    search"; Section 3): point p collides with query q in table l when value_l(p) == value_l(q);
    q's candidates are the distinct ids of every point colliding with it in at least one table.
    Returns (counts int32[m], ids int64[m, max_candidates]): the number of distinct candidates and
    the smallest max_candidates of them in increasing order, padded with -1.  values uint32[n, L],
    ids int64[n], queries uint32[m, L]."""
    values = np.asarray(values, dtype=np.uint32)
    queries = np.asarray(queries, dtype=np.uint32)
    ids = np.asarray(ids, dtype=np.int64)
    L = values.shape[1] if values.ndim == 2 else queries.shape[1]
    tables = [dict() for _ in range(L)]
    for p in range(values.shape[0]):
        for l in range(L):
            tables[l].setdefault(int(values[p, l]), []).append(int(ids[p]))
    m = queries.shape[0]
    counts = np.zeros(m, dtype=np.int32)
    out = np.full((m, max_candidates), -1, dtype=np.int64)
    for q in range(m):
        cand = set()
        for l in range(L):
            cand.update(tables[l].get(int(queries[q, l]), ()))
        c = sorted(cand)
        counts[q] = len(c)
        out[q, :min(len(c), max_candidates)] = c[:max_candidates]
    return counts, out


def weight_class(indptr, weights):
    """Weight class of each set (Section 3, "Bottom-k minhash and fast approximate near neighbor
    search": the data is split into classes ||x||_1 in [2^c, 2^(c+1))): c = floor(log2 ||x||_1),
    where ||x||_1 is the exact sum of the set's positive finite binary32 weights, added as
    Fractions (zero, negative, NaN and infinite weights take no part); a set with no such weight
    gets 0.  Normalising a class to ||x||_1 in [1, 2) means scale = -c."""
    indptr = np.asarray(indptr, dtype=np.int64)
    w = np.asarray(weights, dtype=np.float32)
    out = np.zeros(len(indptr) - 1, dtype=np.int32)
    for s in range(len(out)):
        l1 = Fraction(0)
        for x in w[indptr[s]:indptr[s + 1]].tolist():
            if x > 0 and math.isfinite(x):
                l1 += Fraction(x)          # a binary32 value is exactly a Python float
        if l1 > 0:
            c = l1.numerator.bit_length() - l1.denominator.bit_length()
            while Fraction(2) ** c > l1:
                c -= 1
            while Fraction(2) ** (c + 1) <= l1:
                c += 1
            out[s] = c
    return out


def bottomk(indptr, indices, weights, k: int, seed: int, *, phi0: float = 1.0, threads: int = 1,
            work: bool = False):
    """Bottom-k weighted sketch uint64[n, k] (Section 3): t = k, phi raised until DartHash returns
    at least k darts, the k smallest keys in increasing order (all ones for an empty set)."""
    lib = _load()
    indptr, indices, weights = _csr(indptr, indices, weights)
    n = len(indptr) - 1
    out = np.empty((n, k), dtype=np.uint64)
    wk = np.zeros((n, 4), dtype=np.int64)
    T = _table()

    def fn(a, b):
        ip = indptr[a:b + 1]
        return lib.dmo_bottomk(_ptr(ip), _ptr(indices), _ptr(weights), b - a, k, seed & (2**64 - 1), _ptr(T),
                               float(phi0), ctypes.c_void_p(out.ctypes.data + a * k * 8),
                               ctypes.c_void_p(wk.ctypes.data + a * 32))

    _run_chunked(n, threads, fn)
    return (out, wk) if work else out


def compare(a, c, k: int, bits: int = 0, mode: str = "pairs"):
    """Similarity counts of sketches (Section 1.1, "Similarity estimation"): for each pair, the
    number m of the k minhash slots whose values agree.  bits = 0: rows of k uint64 keys
    (Eq. 1: E[m] = k J); bits = b in {1, 2, 4, 8, 16, 32}: rows of packed b-bit values, slot j at
    bit (j b) mod 64 of word floor(j b / 64) (E[m] = k (J + (1 - J) 2^-b)).  mode "pairs": row i
    of a with row i of c (uint32[n]); "cross": every row of a with every row of c
    (uint32[n_a, n_c]).  Written out slot by slot."""
    a = np.asarray(a, dtype=np.uint64)
    c = np.asarray(c, dtype=np.uint64)

    def values(rows):
        if bits == 0:
            return rows.reshape(len(rows), k)
        out = np.zeros((len(rows), k), dtype=np.uint64)
        mask = np.uint64((1 << bits) - 1)
        for j in range(k):
            word, off = (j * bits) // 64, (j * bits) % 64
            out[:, j] = (rows[:, word] >> np.uint64(off)) & mask
        return out

    va, vc = values(a), values(c)
    if mode == "pairs":
        return (va == vc).sum(axis=1).astype(np.uint32)
    return np.stack([(va[i][None, :] == vc).sum(axis=1) for i in range(len(va))]).astype(np.uint32)


def compare_topk(a, c, k: int, topk: int, bits: int = 0):
    """Top-k neighbours by estimated similarity (Section 1.1, "Similarity estimation": m / k
    estimates J, so the rows with the most agreeing slots are the most similar): for each row i
    of a, the topk rows j of c with the largest count m(i, j) of compare(..., mode="cross"), in
    decreasing order of m, equal m in increasing order of j.  Returns (rows uint32[n_a, topk],
    counts uint32[n_a, topk]); entries past n_c are 0xFFFFFFFF with count 0.  The selection is a
    stable sort of each row of counts."""
    a = np.asarray(a, dtype=np.uint64)
    c = np.asarray(c, dtype=np.uint64)
    n_a = len(a)
    rows = np.full((n_a, topk), 0xFFFFFFFF, dtype=np.uint32)
    counts = np.zeros((n_a, topk), dtype=np.uint32)
    if len(c) == 0:
        return rows, counts
    m = compare(a, c, k, bits, mode="cross").astype(np.int64)
    for i in range(n_a):
        order = np.argsort(-m[i], kind="stable")[:topk]      # stable: equal counts keep row order
        rows[i, :len(order)] = order
        counts[i, :len(order)] = m[i, order]
    return rows, counts


def estimate_jaccard(matches, k: int, bits: int = 0):
    """Weighted Jaccard estimates from agreeing-slot counts m (Section 1.1, "Similarity estimation"):
    m / k for keys, since E[m] = k J (Eq. 1); for b-bit fields E[m] = k (J + (1 - J) 2^-b), which
    solved for J gives (m / k - 2^-b) / (1 - 2^-b).  binary64, one rounding per operation."""
    p = np.asarray(matches, dtype=np.float64) / np.float64(k)
    if bits == 0:
        return p
    r = np.float64(2.0) ** -bits
    return (p - r) / (np.float64(1.0) - r)


DART_DTYPE = np.dtype({
    "names": ["pos", "i", "nu", "rho", "w", "r", "j", "u", "v", "code", "q"],
    "formats": [np.int64, np.uint32, np.int32, np.int32, np.uint64, np.uint64, np.int32,
                np.uint32, np.uint32, np.uint32, np.uint64],
    "offsets": [0, 8, 12, 16, 24, 32, 40, 44, 48, 52, 56],
    "itemsize": 64})


def darthash(indices, weights, t: int, seed: int, theta: float, cap: int = 1 << 20):
    """The kept darts of one row at rank limit theta (Algorithm 1's output set D) plus the
    work counts (areas, darts generated, darts kept)."""
    lib = _load()
    indices = np.ascontiguousarray(indices, dtype=np.uint32)
    weights = np.ascontiguousarray(weights, dtype=np.float32)
    out = np.empty(cap, dtype=DART_DTYPE)
    wk = np.zeros(3, dtype=np.int64)
    n = lib.dmo_darthash(_ptr(indices), _ptr(weights), len(indices), t, seed & (2**64 - 1),
                         _ptr(_table()), float(np.float32(theta)), _ptr(out), cap, _ptr(wk))
    if n < 0:
        raise OracleError(-n)
    assert n <= cap, "increase cap"
    return out[:n].copy(), wk


def mix64(z: int) -> int:
    return int(_load().dmo_mix64(z & (2**64 - 1)))


def fastrange32(h, n):
    return (np.asarray(h, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)
