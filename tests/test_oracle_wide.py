"""Pins of the wide-range oracle (binary64 weights, 64-bit ids; Table 1's norms 2^{+-64},
2^{+-512}) against what the paper and the mathematics fix, independently of its own code:

- its hash equals the C oracle's SplitMix64 (two restatements of the published function);
- the rank code equals the upper half of the binary64 pattern where the rank is a binary64
  number, and brackets the rank everywhere else (Fraction arithmetic);
- on tiny inputs, Algorithm 1's pruned loops give exactly the darts of a brute-force box
  enumeration (exact Fractions, no loop bounds);
- at the norms 2^{+-512}, every visited area meets [0, y] x [0, theta) and the first area
  past each loop bound does not (Fractions), and the kept darts are exactly the darts of the
  visited areas that pass the Fraction tests;
- x <= x' coordinatewise keeps a subset of the darts (Section 2's monotonicity);
- the output does not depend on phi0; a repeated id acts as its largest weight;
- collisions of Section 4's pairs at every norm of Table 1 match the weighted Jaccard
  similarity (Theorem 1);
- invalid and out-of-range inputs give the stated codes."""
import struct
from fractions import Fraction

import numpy as np
import pytest

import workloads
from oracle import wide

T = None


def table():
    global T
    if T is None:
        from oracle import poisson_thresholds
        T = poisson_thresholds()
    return T


def frac(d):
    return Fraction(d[0]) * Fraction(2) ** d[1]


def test_mix64_matches_c_oracle(oracle_mod):
    rng = np.random.default_rng(1)
    for z in [0, 1, 2 ** 64 - 1] + [int(v) for v in rng.integers(0, 2 ** 63, size=200, dtype=np.uint64)]:
        assert wide.mix64(z) == oracle_mod.mix64(z)


def test_rank_code_is_upper_half_of_binary64():
    rng = np.random.default_rng(2)
    for _ in range(3000):
        n = int(rng.integers(1, 2 ** 53))
        e = int(rng.integers(-1070, 960))
        v = float(Fraction(n) * Fraction(2) ** e)              # exact: 53 bits, normal range
        if v < 2.0 ** -1022:
            continue
        bits = struct.unpack(">Q", struct.pack(">d", v))[0]
        assert wide.rank_code((n, e)) == bits >> 32
        assert wide.rank_code((n, e)) == wide._code_of_fraction(Fraction(n) * Fraction(2) ** e)
    assert wide.rank_code((0, 5)) == 0


def test_rank_code_brackets_long_values():
    rng = np.random.default_rng(3)
    for _ in range(2000):
        n = int(rng.integers(1, 2 ** 62)) * (1 << int(rng.integers(0, 900))) + int(rng.integers(0, 2 ** 30))
        e = int(rng.integers(-1500, 100))
        v = Fraction(n) * Fraction(2) ** e
        if not Fraction(2) ** -1022 <= v < Fraction(2) ** 1023:
            continue
        c = wide.rank_code((n, e))
        assert frac(wide.code_value(c)) <= v < frac(wide.code_value(c + 1))
        assert c == wide._code_of_fraction(v)


@pytest.mark.parametrize("x,theta", [(0.3, 0.6), (1.7, 0.45), (2.9, 2.5), (0.05, 5.5), (1.1, 1.0),
                                     (3.4, 13.0)])
def test_pruned_loops_equal_brute_force(x, theta):
    t = 4                                                     # k = 2
    th = wide.dyadic(theta)
    got = {(c, q) + ids[:5] for c, q, ids in wide.element_darts(12345, x, t, wide.seed_key(9), th, table(),
                                                                with_id=True)}
    box = wide.box_darts(12345, x, t, 9, th, 4, 4, table())
    assert t * x < 2 ** 5 - 1 and theta < 2 ** 5 - 1          # the box holds every dart
    assert {b[:7] for b in box} == got
    assert len(got) > 0


@pytest.mark.parametrize("x,theta_e", [(2.0 ** 500 * 1.37, -509), (2.0 ** -520 * 1.9, 510),
                                       (2.0 ** 60 * 1.01, -62), (2.0 ** -70, 58), (0.7, 0)])
def test_loop_bounds_at_extreme_norms(x, theta_e):
    """Every visited area lies partly inside [0, y] x [0, theta), the next column, row, weight
    region and rank region past each bound lie outside, and the kept darts are those of the
    visited areas passing exact tests."""
    t = 1676                                                  # k = 256
    theta = (1_234_567, theta_e - 20)
    th = frac(theta)
    y = Fraction(t) * Fraction(x)
    areas, kept = [], set()
    for c, q, ids in wide.element_darts(77, x, t, wide.seed_key(5), theta, table(), with_id=True, areas=areas):
        kept.add(ids[:5])
    assert areas
    two = Fraction(2)

    def col_edge(nu, rho, w):
        return (2 ** nu - 1) + w * two ** (nu - rho)

    def row_edge(nu, rho, r):
        return (2 ** rho - 1) + r * two ** (rho - nu)

    regions = {}
    for nu, rho, w, r in areas:
        assert col_edge(nu, rho, w) <= y and row_edge(nu, rho, r) < th
        regions.setdefault((nu, rho), {}).setdefault(w, []).append(r)
    nus = {a[0] for a in areas}
    rhos = {a[1] for a in areas}
    nu_top, rho_top = max(nus), max(rhos)
    assert nus == set(range(nu_top + 1)) and rhos == set(range(rho_top + 1))
    assert 2 ** (nu_top + 1) - 1 > y and 2 ** (rho_top + 1) - 1 >= th
    for (nu, rho), cols in regions.items():
        wm = max(cols)
        assert sorted(cols) == list(range(wm + 1))
        assert wm + 1 == 2 ** rho or col_edge(nu, rho, wm + 1) > y
        for w, rows in cols.items():
            rm = max(rows)
            assert sorted(rows) == list(range(rm + 1))
            assert rm + 1 == 2 ** nu or row_edge(nu, rho, rm + 1) >= th
    # kept darts: exact tests on every dart of the visited areas
    e = wide.element_key(wide.seed_key(5), 77)
    expect = set()
    for nu, rho, w, r in areas:
        a = wide.area_key(wide.region_key(e, nu, rho), w, r)
        for j in range(wide.poisson_count(a >> 32, table())):
            d = wide.dart_key(a, j)
            U, V = Fraction(d >> 40, 1 << 24), Fraction((d >> 16) & 0xFFFFFF, 1 << 24)
            if (2 ** nu - 1) + (w + V) * two ** (nu - rho) <= y and (2 ** rho - 1) + (r + U) * two ** (rho - nu) < th:
                expect.add((nu, rho, w, r, j))
    assert kept == expect


def test_monotone_in_weights():
    rng = np.random.default_rng(4)
    t = 331
    for l1 in (2.0 ** 512, 2.0 ** -512, 2.0 ** 64):
        ix, wx = workloads.wide_set(rng, 6, l1)
        wy = wx * rng.uniform(1.0, 1.5, size=6)
        theta = wide.code_value(wide.first_limit_code(1.0, float(wy.sum())))
        for i, a, b in zip(ix, wx, wy):
            sa = {ids[:5] for *_, ids in wide.element_darts(int(i), float(a), t, 11, theta, table(), with_id=True)}
            sb = {ids[:5] for *_, ids in wide.element_darts(int(i), float(b), t, 11, theta, table(), with_id=True)}
            assert sa <= sb


def test_output_independent_of_phi0_and_duplicates():
    rng = np.random.default_rng(5)
    for l1 in (2.0 ** 512, 2.0 ** -512, 1.0):
        ix, wx = workloads.wide_set(rng, 10, l1)
        base = wide.sketch_one(ix, wx, 32, 3, table(), phi0=1.0)
        assert base[0] == 0 and wide.EMPTY not in base[1]
        assert wide.sketch_one(ix, wx, 32, 3, table(), phi0=0.3) == base
        assert wide.sketch_one(ix, wx, 32, 3, table(), phi0=5.0) == base
        # a repeated id with a smaller weight changes nothing
        ix2 = np.concatenate([ix, ix[:3]])
        wx2 = np.concatenate([wx, wx[:3] * 0.5])
        assert wide.sketch_one(ix2, wx2, 32, 3, table())[1] == base[1]


@pytest.mark.parametrize("l1", [2.0 ** 64, 2.0 ** -64, 2.0 ** 512, 2.0 ** -512])
def test_collisions_match_weighted_jaccard(l1):
    """Theorem 1: each bucket of a pair agrees with probability J = b / (2 - b)."""
    rng = np.random.default_rng(6 + int(np.log2(l1)) % 97)
    k, b, pairs = 32, 2 * 0.5 / 1.5, 90
    agree = 0
    for p in range(pairs):
        ix, wx, iy, wy = workloads.wide_pair(rng, 6, b, l1)
        sx = wide.sketch_one(ix, wx, k, 100 + p, table())
        sy = wide.sketch_one(iy, wy, k, 100 + p, table())
        assert sx[0] == 0 and sy[0] == 0
        agree += sum(a == c for a, c in zip(sx[1], sy[1]))
    J, n = b / (2 - b), pairs * k
    assert abs(agree - n * J) <= 4 * np.sqrt(n * J * (1 - J))


def test_errors_and_sentinels():
    T_ = table()
    assert wide.sketch_one([1, 2], [0.5, float("nan")], 8, 1, T_)[0] == wide.EINVAL
    assert wide.sketch_one([1, 2], [0.5, -1.0], 8, 1, T_)[0] == wide.EINVAL
    assert wide.sketch_one([1, 2], [0.5, float("inf")], 8, 1, T_)[0] == wide.EINVAL
    assert wide.sketch_one([1, 2], [0.5, 2.0 ** 960], 8, 1, T_)[0] == wide.ERANGE
    assert wide.sketch_one([1, 2], [2.0 ** 961, float("nan")], 8, 1, T_)[0] == wide.EINVAL
    assert wide.sketch_one([1, 2], [2.0 ** -991, 5e-324], 8, 1, T_)[0] == wide.ERANGE
    st, out = wide.sketch_one([1, 2], [0.0, 0.0], 8, 1, T_)
    assert st == 0 and out == [wide.EMPTY] * 8
    assert wide.sketch_one([], [], 8, 1, T_) == (0, [wide.EMPTY] * 8)
    # subnormal weights beside a normal one, and the largest id
    st, out = wide.sketch_one([2 ** 64 - 1, 3], [5e-324, 1.0], 8, 1, T_)
    assert st == 0 and wide.EMPTY not in out
    # the largest in-range weights (ranks near 2^-990 stay normal)
    st, out = wide.sketch_one([5, 6], [2.0 ** 959, 2.0 ** 958], 8, 1, T_)
    assert st == 0 and wide.EMPTY not in out


def test_one_bit_collisions_match_weighted_jaccard():
    """Section 1.1: a b-bit value agrees with probability J + (1 - J) 2^-b; 1-bit at 2^64."""
    rng = np.random.default_rng(77)
    k, b, pairs = 64, 2 * 0.5 / 1.5, 60
    xs, ys = [], []
    for _ in range(pairs):
        ix, wx, iy, wy = workloads.wide_pair(rng, 6, b, 2.0 ** 64)
        xs.append((ix, wx))
        ys.append((iy, wy))
    bx, by = workloads.wide_csr(xs), workloads.wide_csr(ys)
    wx_, _, sx = wide.sketch_bbit(bx.indptr, bx.indices, bx.weights, k, 1, 5)
    wy_, _, sy = wide.sketch_bbit(by.indptr, by.indices, by.weights, k, 1, 5)
    assert not sx.any() and not sy.any()
    agree = sum(k - bin(int(a) ^ int(c)).count("1") for a, c in zip(wx_[:, 0], wy_[:, 0]))
    J, n = b / (2 - b), pairs * k
    p = J + (1 - J) / 2
    assert abs(agree - n * p) <= 4 * np.sqrt(n * p * (1 - p))


@pytest.mark.parametrize("l1", [2.0 ** 512, 2.0 ** -512, 2.0 ** 64])
def test_kept_dart_count_is_poisson_phi_t(l1):
    """Lemma 1 at Table 1's norms: the darts of rank below theta = phi / ||x||_1 that hit x
    number Poi(phi t) (here t = 331, phi = 1; theta's code truncation lowers phi by < 2^-20)."""
    rng = np.random.default_rng(int(np.log2(l1)) % 1000 + 31)
    t, counts = 331, []
    for s in range(60):
        ix, wx = workloads.wide_set(rng, 8, l1)
        theta = wide.code_value(wide.first_limit_code(1.0, float(wx.sum())))
        counts.append(sum(1 for i, x in zip(ix, wx)
                          for _ in wide.element_darts(int(i), float(x), t, wide.seed_key(1000 + s), theta, table())))
    c = np.array(counts, dtype=float)
    assert abs(c.mean() - t) < 4 * np.sqrt(t / len(c))
    assert 0.6 * t < c.var(ddof=1) < 1.5 * t


def test_darts_per_area_and_uniforms():
    """Algorithm 1's per-area draws under the wide keys: X ~ Poi(1) (chi-square over 0..4+) and
    U, V uniform on [0, 1) (Kolmogorov-Smirnov), over the areas of sets at 2^{+-512}."""
    from math import exp, factorial
    rng = np.random.default_rng(5)
    xs, us, vs = [], [], []
    for l1 in (2.0 ** 512, 2.0 ** -512):
        for s in range(3):
            ix, wx = workloads.wide_set(rng, 8, l1)
            theta = wide.code_value(wide.first_limit_code(1.0, float(wx.sum())))
            areas = []
            for i, x in zip(ix, wx):
                list(wide.element_darts(int(i), float(x), 331, wide.seed_key(s), theta, table(), areas=areas))
                e = wide.element_key(wide.seed_key(s), int(i))
                for nu, rho, w, r in areas:
                    a = wide.area_key(wide.region_key(e, nu, rho), w, r)
                    n = wide.poisson_count(a >> 32, table())
                    xs.append(n)
                    for j in range(n):
                        d = wide.dart_key(a, j)
                        us.append((d >> 40) / 2 ** 24)
                        vs.append(((d >> 16) & 0xFFFFFF) / 2 ** 24)
                areas.clear()
    xs = np.array(xs)
    n = len(xs)
    assert n > 20000
    obs = [np.sum(xs == m) for m in range(4)] + [np.sum(xs >= 4)]
    p = [exp(-1) / factorial(m) for m in range(4)]
    p.append(1 - sum(p))
    chi2 = sum((o - n * q) ** 2 / (n * q) for o, q in zip(obs, p))
    assert chi2 < 18.5                                   # 4 degrees of freedom, p ~ 0.001
    from scipy import stats
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    assert stats.kstest(vs, "uniform").pvalue > 1e-3
