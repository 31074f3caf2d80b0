"""Distributional pins of the oracle (CPU only).

The paper prints no hash values, so the hash-derived bits are pinned by what the method
must satisfy in distribution: Lemma 1's Poisson dart count, Poi(1) darts per area, uniform
positions, consistent weighted sampling marginals, Theorem 1's bucket fill probability,
collision probability = weighted Jaccard (Eq. 1) with independent minhashes, (1 + J)/2 for
1-bit minhash, J^K for (L, K) LSH and the Fig. 2 confidence-interval protocol.  Every test
uses fixed seeds; bounds are 99% (where the spec test asks for it) or |z| < 4.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import workloads

THREADS = 8


def exact_wjaccard(ix, wx, iy, wy):
    a = dict(zip(ix.tolist(), wx.astype(np.float64).tolist()))
    b = dict(zip(iy.tolist(), wy.astype(np.float64).tolist()))
    keys = set(a) | set(b)
    mn = sum(min(a.get(i, 0.0), b.get(i, 0.0)) for i in keys)
    mx = sum(max(a.get(i, 0.0), b.get(i, 0.0)) for i in keys)
    return mn / mx


def pair_batches(pairs):
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])
    return xs, ys


def area_inside(d, y_fr, theta_fr, t):
    """True when dart d's whole area lies below both x_i (weight) and theta (rank)."""
    nu, rho, w, r = int(d["nu"]), int(d["rho"]), int(d["w"]), int(d["r"])
    w_hi = Fraction(2 ** nu - 1) + Fraction(w + 1) * Fraction(2 ** nu, 2 ** rho)
    r_hi = Fraction(2 ** rho - 1) + Fraction(r + 1) * Fraction(2 ** rho, 2 ** nu)
    return w_hi <= y_fr and r_hi <= theta_fr


# ------------------------------------------------------------------------------------------
# Lemma 1 and the dart model
# ------------------------------------------------------------------------------------------
def test_lemma1_kept_darts_are_poisson_phi_t(oracle_mod):
    """DartHash_t(x, phi) returns D ~ Poi(phi t) darts (Lemma 1); with the float limit theta
    the mean is t * ||x||_1 * theta exactly."""
    rng = np.random.default_rng(101)
    t = oracle_mod.t_of_k(64)
    zs, areas, darts = [], 0, 0
    for s in range(500):
        nnz = int(rng.integers(1, 80))
        idx = np.sort(rng.choice(1 << 22, nnz, replace=False)).astype(np.uint32)
        w = (rng.lognormal(size=nnz) * 10 ** rng.uniform(-2, 2)).astype(np.float32)
        l1 = float(w.astype(np.float64).sum())
        phi = float(rng.choice([0.5, 1.0, 2.0]))
        theta = np.float32(phi / l1)
        lam = t * l1 * float(theta)
        _, wk = oracle_mod.darthash(idx, w, t, s, float(theta))
        zs.append((wk[2] - lam) / math.sqrt(lam))
        areas += int(wk[0])
        darts += int(wk[1])
    zs = np.array(zs)
    n = len(zs)
    assert abs(zs.sum() / math.sqrt(n)) < 4                     # mean phi t
    assert abs((np.sum(zs ** 2) - n) / math.sqrt(2 * n)) < 4   # variance phi t
    # every inspected area holds Poi(1) darts: generated ~ Poi(areas)
    assert abs(darts - areas) / math.sqrt(areas) < 4


def test_positions_uniform_inside_areas(oracle_mod):
    """V, U ~ Unif[0, 1) inside each area (Algorithm 1), tested on darts whose area lies
    wholly inside the kept region so the filter does not shape them."""
    rng = np.random.default_rng(7)
    t = oracle_mod.t_of_k(32)
    us, vs = [], []
    for s in range(60):
        idx = np.sort(rng.choice(1 << 20, 20, replace=False)).astype(np.uint32)
        w = (rng.exponential(size=20) * 0.3).astype(np.float32)
        theta = np.float32(3.0 / float(w.sum()))
        darts, _ = oracle_mod.darthash(idx, w, t, s, float(theta))
        th = Fraction(float(theta))
        for d in darts:
            y = Fraction(float(w[int(d["pos"])])) * t
            if area_inside(d, y, th, t):
                us.append(int(d["u"]) / 2 ** 24)
                vs.append(int(d["v"]) / 2 ** 24)
    assert len(us) > 3000
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    assert stats.kstest(vs, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(us, vs)[0, 1]) < 4 / math.sqrt(len(us))


# ------------------------------------------------------------------------------------------
# consistent weighted sampling (Section 1)
# ------------------------------------------------------------------------------------------
def test_winner_element_marginals(oracle_mod):
    """The first dart hitting x lands on element i with probability x_i / ||x||_1: the
    winner of slot j is the element whose singleton set has the same minhash in slot j."""
    w = np.array([0.05, 0.1, 0.2, 0.4, 0.8, 1.6], dtype=np.float32)
    idx = np.array([3, 17, 99, 1000, 4242, 77777], dtype=np.uint32)
    k = 256
    counts = np.zeros(len(w))
    for seed in range(30):
        full = oracle_mod.sketch([0, len(w)], idx, w, k, seed)[0]
        singles = oracle_mod.sketch(np.arange(len(w) + 1), idx, w, k, seed)
        hit = singles == full[None, :]
        assert (hit.sum(axis=0) == 1).all()
        counts += hit.sum(axis=1)
    expected = counts.sum() * w / w.sum()
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert stats.chi2.sf(chi2, len(w) - 1) > 1e-3


def test_winner_weight_uniform_and_min_rank_exponential(oracle_mod):
    """The winning dart's weight is uniform on [0, x_i] (consistent weighted sampling) and
    each bucket's minimum rank is Exp with rate t ||x||_1 / k (Theorem 1's k processes)."""
    rng = np.random.default_rng(9)
    k = 64
    t = oracle_mod.t_of_k(k)
    fr_w, fr_r = [], []
    for s in range(50):
        nnz = 12
        idx = np.sort(rng.choice(1 << 20, nnz, replace=False)).astype(np.uint32)
        w = (rng.exponential(size=nnz) * 10 ** rng.uniform(-1, 1)).astype(np.float32)
        l1 = float(w.astype(np.float64).sum())
        theta = np.float32(6.0 / l1)
        darts, _ = oracle_mod.darthash(idx, w, t, s, float(theta))
        slot = oracle_mod.fastrange32(darts["q"] >> np.uint64(32), k).astype(np.int64)
        key = (darts["code"].astype(np.uint64) << np.uint64(32)) | (darts["q"] & np.uint64(0xFFFFFFFF))
        best = {}
        for n in range(len(darts)):
            j = int(slot[n])
            if j not in best or key[n] < key[best[j]]:
                best[j] = n
        assert len(best) == k
        for j, n in best.items():
            d = darts[n]
            nu, rho, ww, r = int(d["nu"]), int(d["rho"]), int(d["w"]), int(d["r"])
            sw = (2 ** nu - 1) + (ww + int(d["v"]) / 2 ** 24) * 2.0 ** (nu - rho)
            fr_w.append(sw / t / float(w[int(d["pos"])]))
            rank = (2 ** rho - 1) + (r + int(d["u"]) / 2 ** 24) * 2.0 ** (rho - nu)
            fr_r.append(rank * t * l1 / k)
    assert stats.kstest(fr_w, "uniform").pvalue > 1e-3
    assert stats.kstest(fr_r, "expon").pvalue > 1e-3


# ------------------------------------------------------------------------------------------
# Theorem 1: bucket filling
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 8, 64])
def test_fill_probability_at_phi1(oracle_mod, k):
    """With t = ceil(k ln k) + k each bucket holds Poi(t/k) darts at phi = 1, so all k are
    filled with probability (1 - e^{-t/k})^k (0.632 for k = 1, 0.695 for k = 64)."""
    b = workloads.random_sets(4000, 1, 40, 1 << 22, seed=300 + k)
    _, wk = oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 5, work=True, threads=THREADS)
    t = oracle_mod.t_of_k(k)
    p = (1 - math.exp(-t / k)) ** k
    n = len(wk)
    one = int((wk[:, 3] == 1).sum())
    z = (one - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 4, (one / n, p)


def test_coupon_collector_darts_to_fill(oracle_mod):
    """Darts taken in rank order fall in uniform, independent buckets, so the number needed to
    fill all k buckets has mean k H_k (303.6 for k = 64)."""
    rng = np.random.default_rng(31)
    k = 64
    t = oracle_mod.t_of_k(k)
    need = []
    for s in range(300):
        idx = np.sort(rng.choice(1 << 20, 30, replace=False)).astype(np.uint32)
        w = rng.exponential(size=30).astype(np.float32)
        theta = np.float32(4.0 / float(w.sum()))
        darts, _ = oracle_mod.darthash(idx, w, t, 1000 + s, float(theta))
        order = np.argsort(darts["code"], kind="stable")
        slots = oracle_mod.fastrange32(darts["q"][order] >> np.uint64(32), k)
        seen = set()
        for m, j in enumerate(slots.tolist()):
            seen.add(j)
            if len(seen) == k:
                need.append(m + 1)
                break
    hk = sum(1 / i for i in range(1, k + 1))
    var = k * k * sum(1 / i ** 2 for i in range(1, k + 1)) - k * hk
    assert len(need) >= 295
    z = (np.mean(need) - k * hk) / math.sqrt(var / len(need))
    assert abs(z) < 4


# ------------------------------------------------------------------------------------------
# Eq. 1 and the estimators of Section 1.1
# ------------------------------------------------------------------------------------------
def _collisions(oracle_mod, pairs, k, seed):
    xs, ys = pair_batches(pairs)
    a = oracle_mod.sketch(xs.indptr, xs.indices, xs.weights, k, seed, threads=THREADS)
    b = oracle_mod.sketch(ys.indptr, ys.indices, ys.weights, k, seed, threads=THREADS)
    return (a == b).sum(axis=1)


def test_collision_rate_is_weighted_jaccard_99(oracle_mod):
    """Pr[h(x) = h(y)] = J(x, y) (Eq. 1): 10^4 pairs of the paper's pair recipe at J = 0.5,
    k = 64; total collisions inside the binomial 99% interval; per-pair counts dispersed as
    Bin(k, J) (independent minhashes)."""
    rng = np.random.default_rng(2024)
    bpar = 2 * 0.5 / 1.5
    pairs = [workloads.similar_pair(rng, 64, bpar) for _ in range(10_000)]
    J = np.array([exact_wjaccard(*p) for p in pairs])
    k = 64
    c = _collisions(oracle_mod, pairs, k, 77)
    mu = k * J.sum()
    var = k * (J * (1 - J)).sum()
    assert abs(c.sum() - mu) / math.sqrt(var) < 2.576
    disp = (((c - k * J) ** 2) / (k * J * (1 - J))).sum()
    n = len(c)
    vd = 2 + (1 - 6 * J.mean() * (1 - J.mean())) / (k * J.mean() * (1 - J.mean()))
    assert abs(disp - n) / math.sqrt(vd * n) < 4


@pytest.mark.parametrize("target", [0.25, 0.75])
def test_collision_rate_other_similarities(oracle_mod, target):
    rng = np.random.default_rng(int(target * 100))
    bpar = 2 * target / (1 + target)
    pairs = [workloads.similar_pair(rng, 32, bpar) for _ in range(3000)]
    J = np.array([exact_wjaccard(*p) for p in pairs])
    assert abs(J.mean() - target) < 1e-3
    k = 64
    c = _collisions(oracle_mod, pairs, k, 5)
    assert abs(c.sum() - k * J.sum()) / math.sqrt(k * (J * (1 - J)).sum()) < 4


def test_collision_random_overlaps_and_binary_sets(oracle_mod):
    """Random supports with random overlaps and weights across six decades of ||x||_1, and
    0/1 weights, where J is the set Jaccard |A n B| / |A u B|."""
    rng = np.random.default_rng(55)
    pairs = []
    for s in range(3000):
        n = int(rng.integers(1, 60))
        pool = np.sort(rng.choice(1 << 24, 2 * n, replace=False)).astype(np.uint32)
        sx = np.sort(rng.choice(pool, n, replace=False))
        sy = np.sort(rng.choice(pool, n, replace=False))
        if s % 3 == 0:
            wx = np.ones(n, np.float32)
            wy = np.ones(n, np.float32)
        else:
            sc = 10 ** rng.uniform(-3, 3)
            wx = (rng.exponential(size=n) * sc).astype(np.float32)
            wy = wx.copy()
            m = dict(zip(sx.tolist(), wx.tolist()))
            wy = np.array([m.get(i, rng.exponential() * sc) * rng.uniform(0.5, 1.5) for i in sy.tolist()],
                          dtype=np.float32)
        pairs.append((sx, wx, sy, wy))
    J = np.array([exact_wjaccard(*p) for p in pairs])
    for s in range(0, 3000, 3):
        A, B = set(pairs[s][0].tolist()), set(pairs[s][2].tolist())
        assert abs(J[s] - len(A & B) / len(A | B)) < 1e-12
    k = 32
    c = _collisions(oracle_mod, pairs, k, 3)
    assert abs(c.sum() - k * J.sum()) / math.sqrt(k * (J * (1 - J)).sum() + 1e-9) < 4


def test_one_bit_collision_is_one_plus_j_over_two(oracle_mod):
    """1-bit minhash: each bit agrees with probability (1 + J)/2 (Section 1.1)."""
    rng = np.random.default_rng(66)
    bpar = 2 * 0.5 / 1.5
    pairs = [workloads.similar_pair(rng, 48, bpar) for _ in range(3000)]
    J = np.array([exact_wjaccard(*p) for p in pairs])
    xs, ys = pair_batches(pairs)
    k = 128
    a = oracle_mod.sketch_bbit(xs.indptr, xs.indices, xs.weights, k, 1, 8, threads=THREADS)
    b = oracle_mod.sketch_bbit(ys.indptr, ys.indices, ys.weights, k, 1, 8, threads=THREADS)
    diff = np.bitwise_xor(a, b)
    agree = k - np.array([sum(bin(int(v)).count("1") for v in row) for row in diff])
    p = (1 + J) / 2
    assert abs(agree.sum() - k * p.sum()) / math.sqrt(k * (p * (1 - p)).sum()) < 4


def test_lsh_collision_is_j_to_the_k(oracle_mod):
    """(L, K) LSH: a table value collides with probability J^K, independently across the L
    tables (Section 1.2, "Fast similarity search")."""
    rng = np.random.default_rng(88)
    L, K = 32, 3
    bpar = 2 * 0.6 / 1.6
    pairs = [workloads.similar_pair(rng, 40, bpar) for _ in range(1500)]
    J = np.array([exact_wjaccard(*p) for p in pairs])
    xs, ys = pair_batches(pairs)
    a = oracle_mod.lsh(xs.indptr, xs.indices, xs.weights, L, K, 12, threads=THREADS)
    b = oracle_mod.lsh(ys.indptr, ys.indices, ys.weights, L, K, 12, threads=THREADS)
    c = (a == b).sum(axis=1)
    p = J ** K
    assert abs(c.sum() - L * p.sum()) / math.sqrt(L * (p * (1 - p)).sum()) < 4
    disp = (((c - L * p) ** 2) / (L * p * (1 - p))).sum()
    assert abs(disp - len(c)) / math.sqrt(2.2 * len(c)) < 4
    # the LSH output does not depend on the initial phi
    a2 = oracle_mod.lsh(xs.indptr[:201], xs.indices, xs.weights, L, K, 12, phi0=3.0)
    assert (a2 == a[:200]).all()


def test_fig2_protocol_confidence_intervals(oracle_mod):
    """Section 4.1's protocol: for k = 1..100, a fresh pair with J in {0.25, 0.5, 0.75} and a
    fresh seed; the estimate falls in the 95% binomial interval about 95% of the time."""
    rng = np.random.default_rng(4242)
    inside = total = 0
    for target in (0.25, 0.5, 0.75):
        bpar = 2 * target / (1 + target)
        for k in range(1, 101):
            ix, wx, iy, wy = workloads.similar_pair(rng, 50, bpar)
            seed = int(rng.integers(0, 2 ** 62))
            a = oracle_mod.sketch([0, len(ix)], ix, wx, k, seed)[0]
            b = oracle_mod.sketch([0, len(iy)], iy, wy, k, seed)[0]
            c = int((a == b).sum())
            lo, hi = stats.binom.interval(0.95, k, exact_wjaccard(ix, wx, iy, wy))
            inside += lo <= c <= hi
            total += 1
    frac = inside / total
    assert 0.90 <= frac <= 1.0, frac
