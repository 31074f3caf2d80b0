"""GPU parity of dm_sketch_f64 (binary64 weights, 64-bit ids; Table 1's norms) with the wide-range
oracle: identical keys for every set, bucket count and first limit (more retry passes), for sets
at ||x||_1 = 1, 2^{+-64}, 2^{+-512} and between, weights spanning 2^{+-300} within one set,
repeated ids, subnormal weights beside normal ones, zero and empty rows, the largest id, and the
error codes; at Table 1's size (1,024 elements, k = 256) on sampled sets of a batch launched as
the bench launches it."""
import multiprocessing as mp

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

NORMS = [1.0, 2.0 ** 64, 2.0 ** -64, 2.0 ** 512, 2.0 ** -512]


@pytest.fixture(scope="module")
def torch_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def dmx(torch_mod):
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    dmx.load()
    return dmx


def to_dev(torch, b):
    return (torch.from_numpy(np.ascontiguousarray(b.indptr, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.indices, dtype=np.uint64).view(np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.weights, dtype=np.float64)).cuda())


def varied_batch(seed):
    rng = np.random.default_rng(seed)
    rows = []
    for norm in NORMS + [3.7, 2.0 ** -30, 2.0 ** 200]:
        for _ in range(5):
            rows.append(workloads.wide_set(rng, int(rng.integers(1, 40)), norm))
    for _ in range(8):                                   # weights 2^-300 .. 2^300 in one set
        m = int(rng.integers(2, 16))
        rows.append((workloads.wide_ids(rng, m), 2.0 ** rng.uniform(-300, 300, size=m)))
    rows.append((np.array([5, 5, 9], np.uint64), np.array([0.5, 0.25, 0.0])))
    rows.append((np.array([2 ** 64 - 1, 3], np.uint64), np.array([5e-324, 1.0])))
    rows.append((np.array([7], np.uint64), np.array([0.0])))
    rows.append((np.array([], np.uint64), np.array([])))
    rows.append((np.array([1, 2], np.uint64), np.array([2.0 ** 959, 2.0 ** 958])))
    rows.append((np.array([1, 2], np.uint64), np.array([2.0 ** -989, 2.0 ** -1000])))
    rows.append(workloads.wide_set(rng, 70, 2.0 ** -512))   # more than two rounds of 32 lanes
    return workloads.wide_csr(rows)


@pytest.mark.parametrize("k", [1, 7, 64, 256, 1000, 1024])
def test_varied_sets_match_oracle(dmx, torch_mod, k):
    from oracle import wide
    b = varied_batch(100 + k)
    exp, st = wide.sketch(b.indptr, b.indices, b.weights, k, 23)
    assert np.all(st == 0)
    ctx = dmx.dm_create(0)
    for phi0_1024 in (1280, 300):                        # default limit, and one that needs retries
        dmx.dm_set_option(ctx, dmx.OPT_PHI0, phi0_1024)
        got = dmx.dm_sketch_f64(ctx, *to_dev(torch_mod, b), k, 23)
        assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
        assert np.array_equal(got.cpu().numpy().view(np.uint64), exp)
    ctx.close()


@pytest.mark.parametrize("bits", [1, 2, 4, 8, 16, 32])
def test_bbit_words_match_oracle(dmx, torch_mod, bits):
    from oracle import wide
    rng = np.random.default_rng(200 + bits)
    rows = [workloads.wide_set(rng, int(rng.integers(1, 30)), l1) for l1 in NORMS for _ in range(3)]
    rows.append((np.array([4], np.uint64), np.array([0.0])))                      # no positive weight
    rows.append((np.array([8, 9], np.uint64), np.array([0.5, float("nan")])))       # error row
    b = workloads.wide_csr(rows)
    ctx = dmx.dm_create(0)
    for k in (7, 100, 256):
        ew, ek, st = wide.sketch_bbit(b.indptr, b.indices, b.weights, k, bits, 31)
        keys = torch_mod.empty((b.n_sets, k), dtype=torch_mod.int64, device="cuda")
        words = dmx.dm_sketch_f64_bbit(ctx, *to_dev(torch_mod, b), k, bits, 31, out_keys=keys)
        assert dmx.dm_sync_status(ctx, raise_on_error=False) == 1
        assert np.array_equal(words.cpu().numpy().view(np.uint64), ew)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), ek)
    ctx.close()


@pytest.mark.parametrize("weights,code", [([0.5, float("nan")], 1), ([0.5, -1.0], 1), ([float("inf"), 1.0], 1),
                                          ([0.5, 2.0 ** 960], 5), ([2.0 ** -991, 1e-310], 5),
                                          ([2.0 ** 961, float("nan")], 1)])
def test_errors(dmx, torch_mod, weights, code):
    from oracle import wide
    rng = np.random.default_rng(7)
    good = workloads.wide_set(rng, 9, 2.0 ** 64)
    b = workloads.wide_csr([good, (np.array([11, 12], np.uint64), np.array(weights)), good])
    exp, st = wide.sketch(b.indptr, b.indices, b.weights, 16, 3)
    assert list(st) == [0, code, 0]
    ctx = dmx.dm_create(0)
    got = dmx.dm_sketch_f64(ctx, *to_dev(torch_mod, b), 16, 3)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == code
    g = got.cpu().numpy().view(np.uint64)
    assert np.array_equal(g, exp)                        # the failing row holds all ones
    ctx.close()


def _oracle_row(args):
    from oracle import poisson_thresholds, wide
    indices, weights, k, seed = args
    return wide.sketch_one(indices, weights, k, seed, poisson_thresholds())


def test_table1_size_sampled(dmx, torch_mod):
    """Table 1's sets (1,024 elements, k = 256) at each norm, 2,000 sets per norm in one launch;
    the oracle recomputes 2 sampled sets per norm."""
    per, k, seed = 2000, 256, 1
    parts = [workloads.table1_batch(per, 1024, l1, 500 + i) for i, l1 in enumerate(NORMS)]
    b = workloads.WideBatch(np.concatenate([[0]] + [p.indptr[1:] + 1024 * per * i for i, p in enumerate(parts)]),
                            np.concatenate([p.indices for p in parts]), np.concatenate([p.weights for p in parts]))
    rng = np.random.default_rng(3)
    rows = sorted(int(i * per + r) for i in range(len(NORMS)) for r in rng.choice(per, 2, replace=False))
    jobs = [(b.indices[b.indptr[r]:b.indptr[r + 1]], b.weights[b.indptr[r]:b.indptr[r + 1]], k, seed) for r in rows]
    with mp.get_context("spawn").Pool(len(rows)) as pool:
        res = pool.map(_oracle_row, jobs)
    ctx = dmx.dm_create(0)
    got = dmx.dm_sketch_f64(ctx, *to_dev(torch_mod, b), k, seed)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    g = got.cpu().numpy().view(np.uint64)
    ctx.close()
    for r, (st, out) in zip(rows, res):
        assert st == 0
        assert np.array_equal(g[r], np.array(out, dtype=np.uint64))
    assert not np.any(g == np.uint64(2 ** 64 - 1))


def test_counters_and_arguments(dmx, torch_mod):
    b = varied_batch(5)
    ctx = dmx.dm_create(0)
    cnt = torch_mod.zeros(4, dtype=torch_mod.int64, device="cuda")
    dmx.dm_set_option(ctx, dmx.OPT_COUNTERS, cnt.data_ptr())
    dmx.dm_sketch_f64(ctx, *to_dev(torch_mod, b), 64, 1)
    areas, darts, kept, passes = cnt.cpu().tolist()
    assert areas > 0 and darts > 0 and 0 < kept <= darts and passes >= b.n_sets - 2
    dmx.dm_set_option(ctx, dmx.OPT_COUNTERS, 0)
    ip, ix, w = to_dev(torch_mod, b)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_sketch_f64(ctx, ip, ix, w, 1025, 1)
    with pytest.raises(TypeError):
        dmx.dm_sketch_f64(ctx, ip, ix, w.float(), 8, 1)
    ctx.close()
