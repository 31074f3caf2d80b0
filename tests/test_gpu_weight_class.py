"""GPU parity of the weight-class normalised LSH (Section 3): dm_lsh_scaled equals the oracle's
exactly scaled LSH for every set and scale, scale 0 equals dm_lsh, and dm_weight_classes gives
floor(log2 ||x||_1) of the exact norm, equal to the oracle's class for every set."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

THREADS = 16


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


@pytest.mark.parametrize("form", [0, 2])
def test_scaled_lsh_matches_oracle(dmx, torch_mod, oracle_mod, form):
    torch = torch_mod
    b = workloads.random_sets(400, 0, 200, 1 << 22, seed=61, scale_lo=1e-4, scale_hi=1e4)
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_FORM, form)
    ip, ix, w = to_dev(torch, b)
    scale = torch.empty(b.n_sets, dtype=torch.int32, device="cuda")
    cls = dmx.dm_weight_classes(ctx, ip, w, scale_out=scale)
    assert torch.equal(scale, -cls)                     # normalise every class to [1, 2)
    got = dmx.dm_lsh_scaled(ctx, ip, ix, w, 32, 4, 77, scale)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    exp = oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 77, scale=scale.cpu().numpy(), threads=THREADS)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)
    # probing the neighbouring classes of each set (a query's view)
    for d in (-1, 1):
        got = dmx.dm_lsh_scaled(ctx, ip, ix, w, 32, 4, 77, scale + d)
        exp = oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 77, scale=(scale + d).cpu().numpy(),
                             threads=THREADS)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)
    zero = torch.zeros_like(scale)
    assert torch.equal(dmx.dm_lsh_scaled(ctx, ip, ix, w, 32, 4, 77, zero), dmx.dm_lsh(ctx, ip, ix, w, 32, 4, 77))
    ctx.close()


def test_weight_classes(dmx, torch_mod, oracle_mod):
    """Every set's class equals the oracle's exact class bit for bit: random sets over 16 decades,
    the closed-form edge sets (norms at, one unit below and, in binary64, rounding across a power
    of two; subnormals; sums beyond the binary32 range; weights that take no part), large rows,
    and the edge sets again with their elements reversed."""
    import test_oracle_weight_class as pins
    torch = torch_mod
    rand = workloads.random_sets(2000, 0, 100, 1 << 22, seed=62, scale_lo=1e-8, scale_hi=1e8)
    rows = [(rand.indices[rand.indptr[s]:rand.indptr[s + 1]], rand.weights[rand.indptr[s]:rand.indptr[s + 1]])
            for s in range(rand.n_sets)]
    edges = pins.edge_sets()
    for w, _ in edges:
        rows.append((np.arange(len(w), dtype=np.uint32), np.array(w, dtype=np.float32)))
        rows.append((np.arange(len(w), dtype=np.uint32), np.array(w[::-1], dtype=np.float32)))
    rng = np.random.default_rng(63)
    for nnz in (1000, 5000, 40000):                  # many elements per lane and digit
        w = np.float32(2.0) ** rng.integers(-149, 100, size=nnz).astype(np.float32)
        rows.append((np.arange(nnz, dtype=np.uint32), w.astype(np.float32)))
    b = workloads.csr_of(rows)
    ctx = dmx.dm_create(0)
    ip, ix, w = to_dev(torch, b)
    got = dmx.dm_weight_classes(ctx, ip, w).cpu().numpy()
    sc = torch.empty(b.n_sets, dtype=torch.int32, device="cuda")
    dmx.dm_weight_classes(ctx, ip, w, scale_out=sc, norm_exp=2)
    assert np.array_equal(sc.cpu().numpy(), 2 - got)
    ctx.close()
    exp = oracle_mod.weight_class(b.indptr, b.weights)
    assert np.array_equal(got, exp)
    e0 = rand.n_sets
    assert got[e0:e0 + 2 * len(edges):2].tolist() == [c for _, c in edges]


def test_w3s_full_size_sampled(dmx, torch_mod, oracle_mod):
    """The W3S bench workload at full size: exact weight classes of the 1,000,000 W3 sets, each set
    normalised to ||x||_1 in [4, 8) (norm_exp 2), then (64, 8) LSH values, in the bench's form;
    the classes and values of 300 sampled rows, including the first and the last, equal the
    oracle's."""
    torch = torch_mod
    b = workloads.workload3()
    ip, ix, w = to_dev(torch, b)
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    cls = torch.empty(b.n_sets, dtype=torch.int32, device="cuda")
    scl = torch.empty(b.n_sets, dtype=torch.int32, device="cuda")
    dmx.dm_weight_classes(ctx, ip, w, out=cls, scale_out=scl, norm_exp=2)
    got = dmx.dm_lsh_scaled(ctx, ip, ix, w, 64, 8, 1, scl)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    ctx.close()
    assert torch.equal(scl, 2 - cls)
    rng = np.random.default_rng(19)
    sel = np.unique(np.concatenate([rng.choice(b.n_sets, 298, replace=False), [0, b.n_sets - 1]]))
    sub = b.rows(sel)
    assert np.array_equal(cls.cpu().numpy()[sel], oracle_mod.weight_class(sub.indptr, sub.weights))
    exp = oracle_mod.lsh(sub.indptr, sub.indices, sub.weights, 64, 8, 1, scale=scl.cpu().numpy()[sel],
                         threads=THREADS)
    assert np.array_equal(got.cpu().numpy().view(np.uint32)[sel], exp)
