"""GPU parity of the LSH-table index (dm_lsh_index_*) with the oracle's dictionary-based query:
the same distinct-candidate counts and the same smallest candidate ids, for LSH values made by
the library from near-duplicate pairs, for explicit ids over several insert calls, and for the
limits (capacity, buffer overflow)."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


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


def test_index_matches_oracle_on_near_duplicates(dmx, torch_mod, oracle_mod):
    torch = torch_mod
    rng = np.random.default_rng(40)
    L, K = 24, 2
    pairs = [workloads.similar_pair(rng, 20, 2 * 0.6 / 1.6) for _ in range(3000)]
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])
    ctx = dmx.dm_create(0)
    vx = dmx.dm_lsh(ctx, *to_dev(torch, xs), L, K, 9)
    vy = dmx.dm_lsh(ctx, *to_dev(torch, ys), L, K, 9)
    ctx.close()
    ix = dmx.LshIndex(L, 5000)
    ix.insert(vx[:1800])                                   # two batches: ids 0..1799, 1800..2999
    ix.insert(vx[1800:])
    assert ix.size() == 3000
    counts, ids = ix.query(vy, 32)
    assert ix.status() == 0
    ec, eids = oracle_mod.lsh_index_query(vx.cpu().numpy().view(np.uint32), np.arange(3000),
                                          vy.cpu().numpy().view(np.uint32), 32)
    assert np.array_equal(counts.cpu().numpy(), ec)
    assert np.array_equal(ids.cpu().numpy(), eids)
    found = np.mean([i in eids[i] for i in range(3000)])
    assert found > 0.5                                     # most partners are among the candidates
    # every point finds itself
    counts, ids = ix.query(vx, 8)
    assert np.all(counts.cpu().numpy() >= 1)
    ix.close()


def test_index_explicit_ids_and_limits(dmx, torch_mod, oracle_mod):
    torch = torch_mod
    rng = np.random.default_rng(41)
    L = 8
    vals = rng.integers(0, 50, size=(1000, L), dtype=np.uint32)        # many shared values
    ids = rng.choice(10 ** 9, size=1000, replace=False).astype(np.int64)
    q = rng.integers(0, 50, size=(64, L), dtype=np.uint32)
    dv = torch.from_numpy(vals.view(np.int32)).cuda()
    ix = dmx.LshIndex(L, 1000)
    ix.insert(dv, torch.from_numpy(ids).cuda())
    counts, got = ix.query(torch.from_numpy(q.view(np.int32)).cuda(), 100)
    ec, eids = oracle_mod.lsh_index_query(vals, ids, q, 100)
    c = counts.cpu().numpy()
    ok = c >= 0
    assert ok.sum() > 0
    assert np.array_equal(c[ok], ec[ok])
    assert np.array_equal(got.cpu().numpy()[ok], eids[ok])
    # a query gathering more than the 2,048-collision buffer is flagged
    assert np.all((c == -1) == (np.array([sum(int((vals[:, l] == q[i, l]).sum()) for l in range(L))
                                          for i in range(64)]) > 2048))
    with pytest.raises(dmx.DartMinHashError):
        ix.insert(dv[:1])                                  # past the capacity
    ix.close()
