"""Wide-range DartMinHash (binary64 weights, 64-bit element ids) -- ORACLE, test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may import this module.
It shares no code with the CUDA library.  Pure Python integers, exact throughout.

Why a variant.  The paper's experiments hash 64-bit element ids with double-precision weights
and run the norms ||x||_1 = 2^{+-64} and 2^{+-512} (Section 4, "Synthetic data"; Table 1).  The
binary32 method packs an area's (nu, rho, w, r) into one 64-bit counter and codes ranks as
binary32 values; neither reaches regions nu, rho ~ 500 or ranks ~ 2^{+-512}.  This variant
keeps the dart process of Section 2 and Algorithm 1 and changes only what cannot stretch:

- Element ids i are uint64; e_i = M(sigma + gamma (i + 1)) mod 2^64 (as before).
- Area keys are two-level: the region key z = M(e_i + gamma (1 + 2^16 nu + rho)) and the area key
  a = M(z + gamma (1 + 2^32 w + r)), for nu, rho < 2^16 and w, r < 2^32.
- X ~ Poi(1) by inversion of the top 32 bits of a; dart j has d = M(a + gamma (j + 1)),
  U = (d >> 40) / 2^24, V = ((d >> 16) mod 2^24) / 2^24 (as before).  With y = t x_i:
      t * weight = 2^nu - 1 + (w + V) 2^(nu - rho)       hits x iff t * weight <= y
      rank       = 2^rho - 1 + (r + U) 2^(rho - nu)
- The rank code is the upper 32 bits of the binary64 pattern of the rank rounded toward zero
  (sign, 11 exponent bits, 20 fraction bits); the key is (code << 32) | (q mod 2^32) with
  q = M(d xor SLOT_SALT), and the bucket is fastrange(q >> 32, k) (as before).
- Rank limit: theta is a number whose binary64 pattern has zero low 32 bits; a dart is kept iff
  code(rank) < code(theta), i.e. iff rank < theta.  Theorem 1's loop starts at the binary64
  quotient phi0 / ||x||_1 with its low 32 bits cleared and doubles theta (code + 2^20) until
  every bucket holds a dart, for at most 17 passes (else EOVERFLOW).  The cut is made on the
  key's own code, so the output does not depend on theta, ||x||_1 or the schedule.
- Range: a weight >= 2^960, or a row whose largest weight is positive but below 2^-990, is
  rejected (ERANGE): this keeps every rank of a dart that can hit x, and every limit, a normal
  binary64 number.  A column or row index reaching 2^32 is also ERANGE (it needs t phi >= 2^31).
  Negative, NaN or infinite weights are EINVAL; a row without a positive weight gives the
  all-ones sentinel in every bucket.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
SEED_SALT = 0x243F6A8885A308D3
SLOT_SALT = 0x13198A2E03707344
EMPTY = MASK

OK, EINVAL, ERANGE, EOVERFLOW = 0, 1, 5, 6
MAX_PASSES = 17
X_MAX = 2.0 ** 960
X_MIN_MAX = 2.0 ** -990


class WideError(Exception):
    def __init__(self, code: int):
        super().__init__(code)
        self.code = code


# ------------------------------------------------------------------------------------------
# hashing (SplitMix64's output function, Steele, Lea and Flood 2014, used counter-style)
# ------------------------------------------------------------------------------------------
def mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def seed_key(seed: int) -> int:
    return mix64(seed ^ SEED_SALT)


def element_key(sigma: int, i: int) -> int:
    return mix64(sigma + GOLDEN * (i + 1))


def region_key(e: int, nu: int, rho: int) -> int:
    assert 0 <= nu < 1 << 16 and 0 <= rho < 1 << 16
    return mix64(e + GOLDEN * (1 + (nu << 16) + rho))


def area_key(z: int, w: int, r: int) -> int:
    assert 0 <= w < 1 << 32 and 0 <= r < 1 << 32
    return mix64(z + GOLDEN * (1 + (w << 32) + r))


def dart_key(a: int, j: int) -> int:
    return mix64(a + GOLDEN * (j + 1))


def poisson_count(u32: int, T) -> int:
    return sum(1 for n in range(12) if u32 >= int(T[n]))


def fastrange32(h: int, n: int) -> int:
    return (h * n) >> 32


# ------------------------------------------------------------------------------------------
# exact dyadic numbers n * 2^e (Python integers)
# ------------------------------------------------------------------------------------------
def dyadic(x: float):
    n, d = float(x).as_integer_ratio()
    assert d & (d - 1) == 0
    return n, -(d.bit_length() - 1)


def cmp(a, b) -> int:
    """-1, 0, 1 as a <, =, > b for dyadics a = (n, e), b = (n, e)."""
    m = min(a[1], b[1])
    x, y = a[0] << (a[1] - m), b[0] << (b[1] - m)
    return (x > y) - (x < y)


def rank_code(v) -> int:
    """Upper 32 bits of the binary64 pattern of v rounded toward zero (v >= 0, normal or 0)."""
    n, e = v
    if n == 0:
        return 0
    L = n.bit_length()
    E = L - 1 + e                                   # 2^E <= v < 2^(E+1)
    assert -1022 <= E <= 1023
    top = n >> (L - 21) if L >= 21 else n << (21 - L)   # floor(v 2^(20 - E)), 21 bits
    return ((E + 1023) << 20) | (top - (1 << 20))


def code_value(c: int):
    """The number whose binary64 pattern is c << 32 (a normal code)."""
    E = (c >> 20) - 1023
    assert 1 <= (c >> 20) <= 2046
    return (1 << 20) | (c & 0xFFFFF), E - 20


def first_limit_code(phi0: float, l1: float) -> int:
    """Theorem 1's first limit phi0 / ||x||_1 (binary64 quotient) with the low 32 bits cleared."""
    q = np.float64(phi0) / np.float64(l1)
    return int(np.array([q], dtype=np.float64).view(np.uint64)[0]) >> 32


# ------------------------------------------------------------------------------------------
# Algorithm 1 for one element (all darts of rank < theta that hit x)
# ------------------------------------------------------------------------------------------
def element_darts(index: int, x: float, t: int, sigma: int, theta, T, work=None, with_id=False, areas=None):
    """Yields (code, q[, (nu, rho, w, r, j, u, v)]) for every kept dart of element ``index``
    with weight x > 0 under the limit theta (a dyadic).  Loops in Algorithm 1's order
    nu, rho, w, r, j with its loop bounds.  ``areas``: a list that receives every visited
    (nu, rho, w, r)."""
    y = (t * dyadic(x)[0], dyadic(x)[1])                      # t x_i, exact
    e = element_key(sigma, index)
    nu = 0
    while cmp(((1 << nu) - 1, 0), y) <= 0:                     # 2^nu - 1 <= y
        rho = 0
        while cmp(((1 << rho) - 1, 0), theta) < 0:             # 2^rho - 1 < theta
            # a column or row index 2^32 would be visited: outside the area key's range
            if rho > 32 and cmp(((((1 << nu) - 1) << rho) + ((1 << 32) << nu), -rho), y) <= 0:
                raise WideError(ERANGE)
            if nu > 32 and cmp(((((1 << rho) - 1) << nu) + ((1 << 32) << rho), -nu), theta) < 0:
                raise WideError(ERANGE)
            z = region_key(e, nu, rho)
            w = 0
            # column w's left edge 2^nu - 1 + w 2^(nu - rho) must be <= y
            while w < (1 << rho) and cmp(((((1 << nu) - 1) << rho) + (w << nu), -rho), y) <= 0:
                r = 0
                # row r's lower edge 2^rho - 1 + r 2^(rho - nu) must be < theta
                while r < (1 << nu) and cmp(((((1 << rho) - 1) << nu) + (r << rho), -nu), theta) < 0:
                    if areas is not None:
                        areas.append((nu, rho, w, r))
                    a = area_key(z, w, r)
                    X = poisson_count(a >> 32, T)
                    if work is not None:
                        work[0] += 1
                        work[1] += X
                    for j in range(X):
                        d = dart_key(a, j)
                        u, v = d >> 40, (d >> 16) & 0xFFFFFF
                        tw = ((((1 << nu) - 1) << (rho + 24)) + (((w << 24) | v) << nu), -(rho + 24))
                        rank = ((((1 << rho) - 1) << (nu + 24)) + (((r << 24) | u) << rho), -(nu + 24))
                        if cmp(tw, y) > 0 or cmp(rank, theta) >= 0:
                            continue
                        if work is not None:
                            work[2] += 1
                        q = mix64(d ^ SLOT_SALT)
                        if with_id:
                            yield rank_code(rank), q, (nu, rho, w, r, j, u, v)
                        else:
                            yield rank_code(rank), q
                    r += 1
                w += 1
            rho += 1
        nu += 1


def check_row(weights) -> tuple[int, float]:
    """(status, ||x||_1 as a binary64 sum in row order).  An invalid weight anywhere in the row
    gives EINVAL, before any range check."""
    ws = [float(x) for x in weights]
    if any(not (x >= 0.0) or x == float("inf") for x in ws):
        return EINVAL, 0.0
    if any(x >= X_MAX for x in ws):
        return ERANGE, 0.0
    mx = max(ws, default=0.0)
    if 0.0 < mx < X_MIN_MAX:
        return ERANGE, 0.0
    l1 = 0.0
    for x in ws:
        l1 += x
    return OK, l1


def sketch_one(indices, weights, k: int, seed: int, T, phi0: float = 1.0, work=None):
    """Theorem 1: the k minhash keys of one set.  Returns (status, keys)."""
    from . import t_of_k
    t = t_of_k(k)
    out = [EMPTY] * k
    st, l1 = check_row(weights)
    if st:
        return st, out
    if l1 == 0.0:
        return OK, out
    sigma = seed_key(seed)
    c = first_limit_code(phi0, l1)
    for p in range(MAX_PASSES):
        theta = code_value(c)
        out = [EMPTY] * k
        try:
            for i, x in zip(indices, weights):
                if float(x) > 0.0:
                    for code, q in element_darts(int(i), float(x), t, sigma, theta, T, work):
                        key = (code << 32) | (q & 0xFFFFFFFF)
                        j = fastrange32(q >> 32, k)
                        if key < out[j]:
                            out[j] = key
        except WideError as err:
            return err.code, [EMPTY] * k
        if work is not None:
            work[3] += 1
        if all(v != EMPTY for v in out):
            return OK, out
        c += 1 << 20
    return EOVERFLOW, [EMPTY] * k


def sketch(indptr, indices, weights, k: int, seed: int, phi0: float = 1.0, sets=None):
    """Keys uint64[n, k] (rows of sets with an error hold the sentinel) and per-set status.
    ``sets``: optional subset of row numbers to compute (others stay sentinel, status -1)."""
    from . import poisson_thresholds
    T = poisson_thresholds()
    n = len(indptr) - 1
    out = np.full((n, k), EMPTY, dtype=np.uint64)
    status = np.full(n, -1, dtype=np.int32)
    for s in (range(n) if sets is None else sets):
        b, e = int(indptr[s]), int(indptr[s + 1])
        st, keys = sketch_one(indices[b:e], weights[b:e], k, seed, T, phi0)
        status[s] = st
        out[s] = np.array(keys, dtype=np.uint64)
    return out, status


# ------------------------------------------------------------------------------------------
# brute force over a bounding box (no loop bounds, no early breaks)
# ------------------------------------------------------------------------------------------
def box_darts(index: int, x: float, t: int, seed: int, theta, nu_box: int, rho_box: int, T):
    """Every dart of element ``index`` in regions nu <= nu_box, rho <= rho_box (all columns, all
    rows) that hits weight x and has rank < theta: a set of (code, q, nu, rho, w, r, j)."""
    from fractions import Fraction
    y = Fraction(t) * Fraction(x)
    th = Fraction(theta[0]) * Fraction(2) ** theta[1]
    e = element_key(seed_key(seed), index)
    found = set()
    for nu in range(nu_box + 1):
        for rho in range(rho_box + 1):
            z = region_key(e, nu, rho)
            for w in range(1 << rho):
                for r in range(1 << nu):
                    a = area_key(z, w, r)
                    for j in range(poisson_count(a >> 32, T)):
                        d = dart_key(a, j)
                        U = Fraction(d >> 40, 1 << 24)
                        V = Fraction((d >> 16) & 0xFFFFFF, 1 << 24)
                        tw = (2 ** nu - 1) + (w + V) * Fraction(2) ** (nu - rho)
                        rank = (2 ** rho - 1) + (r + U) * Fraction(2) ** (rho - nu)
                        if tw <= y and rank < th:
                            found.add((_code_of_fraction(rank), mix64(d ^ SLOT_SALT), nu, rho, w, r, j))
    return found


def _code_of_fraction(v) -> int:
    """rank_code restated on a Fraction: exponent by search, then floor(v / 2^(E - 20))."""
    from fractions import Fraction
    if v == 0:
        return 0
    E = v.numerator.bit_length() - v.denominator.bit_length()
    while Fraction(2) ** E > v:
        E -= 1
    while Fraction(2) ** (E + 1) <= v:
        E += 1
    top = int(v / Fraction(2) ** (E - 20))
    assert (1 << 20) <= top < (1 << 21)
    return ((E + 1023) << 20) | (top - (1 << 20))


# ------------------------------------------------------------------------------------------
# b-bit minhash (Section 1.1, "Similarity estimation") of the wide-range keys
# ------------------------------------------------------------------------------------------
BBIT_SALT = 0xA4093822299F31D0


def sketch_bbit(indptr, indices, weights, k: int, b: int, seed: int, phi0: float = 1.0):
    """(words uint64[n, ceil(k b / 64)], keys uint64[n, k], status): each minhash is mapped to
    the low b bits of M(key xor BBIT_SALT); slot j sits at bit (j b) mod 64 of word
    floor(j b / 64), least significant bit first.  Rows of sets with an error are all ones."""
    assert b in (1, 2, 4, 8, 16, 32)
    keys, status = sketch(indptr, indices, weights, k, seed, phi0)
    n, W = len(indptr) - 1, (k * b + 63) // 64
    words = np.zeros((n, W), dtype=np.uint64)
    for s in range(n):
        if status[s]:
            words[s] = np.uint64(MASK)
            continue
        row = [0] * W
        for j in range(k):
            beta = mix64(int(keys[s, j]) ^ BBIT_SALT) & ((1 << b) - 1)
            row[(j * b) // 64] |= beta << ((j * b) % 64)
        words[s] = np.array(row, dtype=np.uint64)
    return words, keys, status
