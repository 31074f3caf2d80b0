"""Data-parallel split across processes: two ranks (a gloo group, as bench.py sets up for N > 1)
each sketch their own shard of a batch through their own context, gather the keys to rank 0 with
a collective, and the gathered rows equal the oracle's keys of the whole batch.  Both ranks run
on cuda:0 here (one GPU in this environment); their kernels never wait on one another, so the
result is the same as on two GPUs."""
import os
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_SETS, K, SEED = 600, 256, 5


def _batch():
    return workloads.random_sets(N_SETS, 1, 300, 1 << 24, seed=71)


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch

    import bench
    import paper_2005_11547_gb300 as dmx
    try:
        r, w, _ = bench.dist_env()
        dist = bench.dist_init(w, use_cuda=False)
        torch.cuda.set_device(0)
        dmx.load()
        b = _batch()
        lo, hi = r * N_SETS // w, (r + 1) * N_SETS // w
        sub = b.rows(range(lo, hi))
        ip = torch.from_numpy(sub.indptr).cuda()
        ix = torch.from_numpy(sub.indices.view(np.int32)).cuda()
        wt = torch.from_numpy(sub.weights).cuda()
        ctx = dmx.dm_create(0)
        keys = dmx.dm_sketch(ctx, ip, ix, wt, K, SEED)
        dmx.dm_sync_status(ctx)
        ctx.close()
        parts = [torch.empty((N_SETS // w, K), dtype=torch.int64) for _ in range(w)]
        dist.all_gather(parts, keys.cpu())
        bench.barrier(dist, use_cuda=False)
        if r == 0:
            q.put(torch.cat(parts).numpy().view(np.uint64).copy())
        dist.destroy_process_group()
    except Exception as e:                      # reported to the parent
        q.put(repr(e))
        raise


def test_two_ranks_sketch_shards_and_gather(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() + 500) % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = q.get(timeout=300)
    finally:
        for p in procs:                         # a rank left waiting in a collective is ended
            p.join(timeout=120)
            if p.is_alive():
                p.kill()
                p.join()
    assert all(p.exitcode == 0 for p in procs)
    assert not isinstance(got, str), got
    b = _batch()
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, K, SEED, threads=8)
    assert got.shape == exp.shape
    assert np.array_equal(got, exp)
