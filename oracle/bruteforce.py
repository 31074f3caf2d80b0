"""Brute-force enumeration of the hashed Poisson dart process -- test infrastructure only.

This is the plain definition the oracle's Algorithm 1 loop must reproduce, written without
any of Algorithm 1's loop bounds or early breaks: for every element, EVERY area of every
region (nu, rho) inside a bounding box nu <= nu_box, rho <= rho_box is visited
(Section 2, "Poisson darts": region (nu, rho) covers weights [(2^nu - 1)/t, (2^(nu+1) - 1)/t)
and ranks [2^rho - 1, 2^(rho+1) - 1), split into 2^rho columns and 2^nu rows), its Poisson
count is drawn, and each dart's weight and rank are evaluated with exact ``Fraction``
arithmetic from the formulas of Algorithm 1:

    weight = W + (w + V) delta_nu,   W = (2^nu - 1)/t,  delta_nu = 2^nu / (t 2^rho)
    rank   = R + (r + U) delta_rho,  R = 2^rho - 1,     delta_rho = 2^rho / 2^nu

A dart hits x iff weight <= x_i.  Minhash j (Theorem 1) is the smallest key among darts in
bucket j.  The box holds every dart of rank < 2^(rho_box+1) - 1, so for every bucket whose
box minimum has a rank below that bound the box minimum is the global minimum.

The hash (SplitMix64's output function, Steele, Lea and Flood 2014, used counter-style) is
written out again here, independently of dm_oracle.c.
"""
from __future__ import annotations

from fractions import Fraction

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
SEED_SALT = 0x243F6A8885A308D3
SLOT_SALT = 0x13198A2E03707344


def mix64(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def rz_binary32_bits(x: Fraction) -> int:
    """Bit pattern of the largest IEEE binary32 value <= x (x >= 0, normal range)."""
    if x == 0:
        return 0
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    assert Fraction(2) ** e <= x < Fraction(2) ** (e + 1)
    assert -126 <= e <= 127
    m = int(x / Fraction(2) ** (e - 23))          # floor: 24-bit significand
    assert 2 ** 23 <= m < 2 ** 24
    return ((e + 127) << 23) | (m - 2 ** 23)


def poisson_count(u32: int, T) -> int:
    return sum(1 for n in range(12) if u32 >= int(T[n]))


def box_darts(index: int, x: float, t: int, seed: int, nu_box: int, rho_box: int, T,
              with_id: bool = False):
    """Every dart of element ``index`` inside the box that hits weight ``x``:
    yields (rank Fraction, key, q), plus (nu, rho, w, r, j) when ``with_id``."""
    sigma = mix64(seed ^ SEED_SALT)
    e = mix64(sigma + GOLDEN * (index + 1))
    xt = Fraction(x) * t                                   # exact: float -> Fraction
    for nu in range(nu_box + 1):
        for rho in range(rho_box + 1):
            W = Fraction(2 ** nu - 1, t)
            R = Fraction(2 ** rho - 1)
            d_nu = Fraction(2 ** nu, t * 2 ** rho)
            d_rho = Fraction(2 ** rho, 2 ** nu)
            for w in range(2 ** rho):
                for r in range(2 ** nu):
                    pack = (nu << 58) | (rho << 52) | (w << nu) | r
                    a = mix64(e + GOLDEN * (pack + 1))
                    X = poisson_count(a >> 32, T)
                    for j in range(X):
                        d = mix64(a + GOLDEN * (j + 1))
                        U = Fraction(d >> 40, 2 ** 24)
                        V = Fraction((d >> 16) & 0xFFFFFF, 2 ** 24)
                        weight = W + (w + V) * d_nu
                        rank = R + (r + U) * d_rho
                        if weight * t <= xt:
                            q = mix64(d ^ SLOT_SALT)
                            key = (rz_binary32_bits(rank) << 32) | (q & 0xFFFFFFFF)
                            if with_id:
                                yield rank, key, q, (nu, rho, w, r, j)
                            else:
                                yield rank, key, q


def sketch(indices, weights, k: int, t: int, seed: int, nu_box: int, rho_box: int, T):
    """Box-limited minhash keys: list of k keys, None where the box holds no dart of rank
    below 2^(rho_box+1) - 1 in that bucket."""
    bound = Fraction(2 ** (rho_box + 1) - 1)
    for x in weights:
        assert Fraction(float(x)) * t < 2 ** (nu_box + 1) - 1, "box too small in weight"
    best = [None] * k
    for i, x in zip(indices, weights):
        if not x > 0:
            continue
        for rank, key, q in box_darts(int(i), float(x), t, seed, nu_box, rho_box, T):
            if rank >= bound:
                continue
            slot = ((q >> 32) * k) >> 32
            if best[slot] is None or key < best[slot]:
                best[slot] = key
    return best


def bottomk(indices, weights, k: int, t: int, seed: int, nu_box: int, rho_box: int, T):
    """Box-limited bottom-k sketch (Section 3, "Bottom-k minhash"): the k smallest keys of the
    darts of rank below 2^(rho_box+1) - 1 that hit x, in increasing order, or None when the box
    holds fewer than k of them (then the box cannot decide the k-th)."""
    bound = Fraction(2 ** (rho_box + 1) - 1)
    for x in weights:
        assert Fraction(float(x)) * t < 2 ** (nu_box + 1) - 1, "box too small in weight"
    keys = []
    for i, x in zip(indices, weights):
        if not x > 0:
            continue
        keys.extend(key for rank, key, q in box_darts(int(i), float(x), t, seed, nu_box, rho_box, T)
                    if rank < bound)
    keys.sort()
    return keys[:k] if len(keys) >= k else None
