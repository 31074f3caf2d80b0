"""GPU parity of dm_lsh ((L, K) LSH values, uint32, bit-exact) with the oracle."""
import numpy as np
import pytest

import workloads
from test_gpu_sketch import assert_same, to_dev  # noqa: F401  (shared helpers)

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


@pytest.fixture(scope="module")
def ctx(dmx):
    c = dmx.dm_create(0)
    yield c
    c.close()


def gpu_lsh(dmx, torch, ctx, b, L, K, seed):
    ip, ix, w = to_dev(torch, b)
    out = dmx.dm_lsh(ctx, ip, ix, w, L, K, seed)
    rc = dmx.dm_sync_status(ctx, raise_on_error=False)
    return out.cpu().numpy().view(np.uint32), rc


@pytest.mark.parametrize("L,K", [(1, 1), (8, 2), (16, 4), (64, 8), (33, 3), (100, 5), (7, 16), (1024, 2),
                                 (700, 32)])
def test_lsh_parity_random_sets(dmx, torch_mod, ctx, oracle_mod, L, K):
    """Ragged sets with ||x||_1 over six decades (both kernels), several (L, K)."""
    b = workloads.random_sets(200, 0, 200, 1 << 24, seed=100 + L + K)
    got, rc = gpu_lsh(dmx, torch_mod, ctx, b, L, K, 77)
    assert rc == 0
    exp = oracle_mod.lsh(b.indptr, b.indices, b.weights, L, K, 77, threads=THREADS)
    assert_same(got, exp, f"L={L} K={K}")


def test_lsh_edge_cases(dmx, torch_mod, ctx, oracle_mod):
    f = np.float32
    rows = [([], []), ([3, 4], [0.0, 0.0]), ([7], [1.0]), ([1, 2, 3], [0.0, 0.5, 0.0]),
            ([5, 5, 5], [0.25, 0.75, 0.5]), ([5], [0.75]), ([9], [3e8]), ([9, 10], [1e-5, 2e-5])]
    b = workloads.csr_of([(np.array(i, np.uint32), np.array(w, f)) for i, w in rows])
    for L, K in [(64, 8), (4, 1), (16, 3)]:
        got, rc = gpu_lsh(dmx, torch_mod, ctx, b, L, K, 5)
        assert rc == 0
        assert_same(got, oracle_mod.lsh(b.indptr, b.indices, b.weights, L, K, 5), f"L={L} K={K}")
    assert (got[0] == 0xFFFFFFFF).all() and (got[1] == 0xFFFFFFFF).all()
    # unlike the minimum, a bottom-K sees a repeated index's darts once per occurrence
    assert not (got[4] == got[5]).all()


def test_lsh_phi0_does_not_change_bits(dmx, torch_mod, ctx):
    b = workloads.random_sets(300, 1, 300, 1 << 24, seed=9)
    ref, _ = gpu_lsh(dmx, torch_mod, ctx, b, 64, 8, 3)
    for v in (1024, 2048, 3000, 16384):
        c2 = dmx.dm_create(0)
        dmx.dm_set_option(c2, 5, v)                 # DM_OPT_LSH_PHI0
        got, rc = gpu_lsh(dmx, torch_mod, c2, b, 64, 8, 3)
        c2.close()
        assert rc == 0
        assert_same(got, ref, f"phi0={v / 1024}")


@pytest.mark.parametrize("form", [1, 2])
def test_lsh_forms(dmx, torch_mod, ctx, form):
    b = workloads.random_sets(300, 0, 300, 1 << 24, seed=19)
    ref, _ = gpu_lsh(dmx, torch_mod, ctx, b, 32, 4, 8)
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_FORM, form)
    got, rc = gpu_lsh(dmx, torch_mod, c2, b, 32, 4, 8)
    c2.close()
    assert rc == 0
    assert_same(got, ref, f"form {form}")


def test_lsh_rejects_oversized_buckets(dmx, torch_mod, ctx):
    b = workloads.random_sets(4, 1, 10, 1 << 20, seed=1)
    with pytest.raises(dmx.DartMinHashError):
        gpu_lsh(dmx, torch_mod, ctx, b, 1024, 32, 1)


def test_w3_full_size_sampled(dmx, torch_mod, ctx, oracle_mod):
    """W3 at full size (1,000,000 tf-idf-like sets, L = 64, K = 8), 500 sampled rows."""
    b = workloads.workload3()
    got, rc = gpu_lsh(dmx, torch_mod, ctx, b, 64, 8, 1)
    assert rc == 0
    rng = np.random.default_rng(3)
    sel = np.unique(np.concatenate([rng.choice(b.n_sets, 495, replace=False), [0, b.n_sets - 1]]))
    sub = b.rows(sel)
    exp = oracle_mod.lsh(sub.indptr, sub.indices, sub.weights, 64, 8, 1, threads=THREADS)
    assert_same(got[sel], exp, "W3")
