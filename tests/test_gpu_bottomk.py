"""GPU parity of dm_bottomk (bottom-k weighted sketch, Section 3) with the oracle: bit-exact
uint64 keys in increasing order, over ragged batches, norms over many decades, every k class
(k within one bitonic buffer size up to the 1024 maximum), the launch forms, the autotuner and
graph replay."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

THREADS = 16
U64MAX = np.uint64(2 ** 64 - 1)


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
            torch.from_numpy(np.ascontiguousarray(b.indices, dtype=np.uint32).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.weights, dtype=np.float32)).cuda())


def run(dmx, torch, ctx, b, k, seed):
    ip, ix, w = to_dev(torch, b)
    out = dmx.dm_bottomk(ctx, ip, ix, w, k, seed)
    rc = dmx.dm_sync_status(ctx, raise_on_error=False)
    return out.cpu().numpy().view(np.uint64), rc


def assert_same(got, exp, what):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        r, c = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches; first row {r} col {c}: "
                             f"gpu {int(got[r, c]):016x} oracle {int(exp[r, c]):016x}")


@pytest.mark.parametrize("k", [1, 7, 32, 64, 100, 256, 1000, 1024])
def test_bottomk_parity_ragged(dmx, torch_mod, oracle_mod, k):
    b = workloads.random_sets(250, 0, 300, 1 << 24, seed=300 + k)
    ctx = dmx.dm_create(0)
    got, rc = run(dmx, torch_mod, ctx, b, k, 4242)
    ctx.close()
    assert rc == 0
    assert_same(got, oracle_mod.bottomk(b.indptr, b.indices, b.weights, k, 4242, threads=THREADS), f"k={k}")


def test_bottomk_extreme_norms_and_edges(dmx, torch_mod, oracle_mod):
    rng = np.random.default_rng(9)
    rows = [(np.zeros(0, np.uint32), np.zeros(0, np.float32)),
            (np.array([5], np.uint32), np.array([1.0], np.float32)),
            (np.array([1, 2], np.uint32), np.array([0.0, 0.0], np.float32)),
            (np.array([3, 4, 5], np.uint32), np.array([1e-30, 2.0, 0.0], np.float32))]
    for s in range(120):
        nnz = int(rng.integers(1, 80))
        idx = np.sort(rng.choice(1 << 24, nnz, replace=False)).astype(np.uint32)
        z = rng.lognormal(size=nnz)
        rows.append((idx, (z / z.sum() * 10 ** rng.uniform(-5, 5)).astype(np.float32)))
    b = workloads.csr_of(rows)
    ctx = dmx.dm_create(0)
    for k in (16, 300):
        got, rc = run(dmx, torch_mod, ctx, b, k, 11)
        assert rc == 0
        exp = oracle_mod.bottomk(b.indptr, b.indices, b.weights, k, 11, threads=THREADS)
        assert_same(got, exp, f"k={k}")
        assert np.all(got[0] == U64MAX) and np.all(got[2] == U64MAX)
    ctx.close()


@pytest.mark.parametrize("form", [0, 1, 2])
def test_bottomk_forms(dmx, torch_mod, oracle_mod, form):
    b = workloads.workload2(800)
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_FORM, form)
    got, rc = run(dmx, torch_mod, ctx, b, 128, 6)
    ctx.close()
    assert rc == 0
    assert_same(got, oracle_mod.bottomk(b.indptr, b.indices, b.weights, 128, 6, threads=THREADS), f"form {form}")


def test_bottomk_w1_prefix_autotune_graph(dmx, torch_mod, oracle_mod):
    """20,000 W1 sets, k = 256: the autotuner's choice and graph replay keep the bits."""
    torch = torch_mod
    b = workloads.workload1(20_000)
    ip, ix, w = to_dev(torch, b)
    ctx = dmx.dm_create(0)
    before = dmx.dm_bottomk(ctx, ip, ix, w, 256, 1)
    dmx.dm_autotune(ctx, ip, ix, w, 256, 1, bottomk=True)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    for _ in range(2):
        after = dmx.dm_bottomk(ctx, ip, ix, w, 256, 1)
        assert torch.equal(before, after)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    ctx.close()
    exp = oracle_mod.bottomk(b.indptr, b.indices, b.weights, 256, 1, threads=THREADS)
    assert_same(after.cpu().numpy().view(np.uint64), exp, "W1 prefix")


def test_w1b_full_size_sampled(dmx, torch_mod, oracle_mod):
    """The W1B bench workload at full size (bottom-k sketches, k = 256, of the 1,000,000 W1 sets)
    in the bench's launch configuration (autotuned, graph replay): 300 sampled rows, including
    the first and the last, equal the oracle's."""
    torch = torch_mod
    b = workloads.workload1()
    ip, ix, w = to_dev(torch, b)
    ctx = dmx.dm_create(0)
    dmx.dm_autotune(ctx, ip, ix, w, 256, 1, bottomk=True)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    out = dmx.dm_bottomk(ctx, ip, ix, w, 256, 1)
    again = dmx.dm_bottomk(ctx, ip, ix, w, 256, 1)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    assert torch.equal(out, again)
    ctx.close()
    rng = np.random.default_rng(17)
    sel = np.unique(np.concatenate([rng.choice(b.n_sets, 298, replace=False), [0, b.n_sets - 1]]))
    sub = b.rows(sel)
    exp = oracle_mod.bottomk(sub.indptr, sub.indices, sub.weights, 256, 1, threads=THREADS)
    assert_same(out.cpu().numpy().view(np.uint64)[sel], exp, "W1B")


def test_bottomk_rejects_bad_k(dmx, torch_mod):
    b = workloads.random_sets(10, 1, 10, 1000, seed=2)
    ctx = dmx.dm_create(0)
    ip, ix, w = to_dev(torch_mod, b)
    for k in (0, 1025):
        with pytest.raises(dmx.DartMinHashError):
            dmx.dm_bottomk(ctx, ip, ix, w, k, 1)
    ctx.close()
