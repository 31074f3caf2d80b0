"""The checked build (libdartminhash_checked.so: every kernel also checks its shared-memory ring,
table and bucket indices) on the paths the product runs: batched, plain and persistent forms
with the block-per-set class, both slot layouts, the general walk, LSH, bottom-k, k = 8192 and
the allocation-free entry.  No check fails (dm_sync_status would return DM_ECHECK) and every
output equals the oracle's.  The library is loaded in a process of its own, so the product
library of the other tests is untouched."""
import os
import sys

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
THREADS = 16


def _batches():
    rng = np.random.default_rng(66)
    rows = []
    for _ in range(300):
        nnz = int(min(5000, max(1, np.exp(np.log(60) + 1.5 * rng.standard_normal()))))
        idx = np.sort(rng.choice(1 << 24, nnz, replace=False)).astype(np.uint32)
        z = rng.lognormal(size=nnz)
        rows.append((idx, (z / z.sum() * 10 ** rng.uniform(-3, 3)).astype(np.float32)))
    return {"w0": workloads.workload0(1000), "heavy": workloads.csr_of(rows),
            "small": workloads.random_sets(40, 1, 300, 1 << 24, seed=9)}


def _cases():
    """(name, batch, call, k, K or 0, form, slots)."""
    out = [("w0", "w0", "sketch", 64, 0, 0, 0)]
    for form in (0, 1, 2):
        for slots in (1, 2):
            for k in (64, 1024):
                out.append((f"heavy f{form} s{slots} k{k}", "heavy", "sketch", k, 0, form, slots))
    out += [("lsh 64x8", "heavy", "lsh", 64, 8, 0, 0), ("lsh 33x3", "heavy", "lsh", 33, 3, 2, 0),
            ("bottomk 128", "heavy", "bottomk", 128, 0, 0, 0), ("k 8192", "small", "sketch", 8192, 0, 0, 0),
            ("noalloc 256", "heavy", "noalloc", 256, 0, 0, 0)]
    return out


def _worker(q):
    sys.path.insert(0, ROOT)
    try:
        import torch

        import paper_2005_11547_gb300 as dmx
        dmx.load(dmx.LIB_CHECKED)
        assert dmx.dm_build_flags() & 1
        batches = _batches()
        res = {}
        for name, bn, call, k, K, form, slots in _cases():
            b = batches[bn]
            ip = torch.from_numpy(b.indptr).cuda()
            ix = torch.from_numpy(b.indices.view(np.int32)).cuda()
            w = torch.from_numpy(b.weights).cuda()
            ctx = dmx.dm_create(0)
            dmx.dm_set_option(ctx, dmx.OPT_FORM, form)
            dmx.dm_set_option(ctx, dmx.OPT_SLOTS, slots)
            dmx.dm_set_option(ctx, dmx.OPT_LARGE_NNZ, 500)
            if call == "sketch":
                out = dmx.dm_sketch(ctx, ip, ix, w, k, 7)
            elif call == "lsh":
                out = dmx.dm_lsh(ctx, ip, ix, w, k, K, 7)
            elif call == "bottomk":
                out = dmx.dm_bottomk(ctx, ip, ix, w, k, 7)
            else:
                out = torch.empty((b.n_sets, k), dtype=torch.int64, device="cuda")
                dmx.dm_sketch_noalloc(ip, ix, w, k, 7, out)
            rc = dmx.dm_sync_status(ctx, raise_on_error=False)
            ctx.close()
            res[name] = (rc, out.cpu().numpy().copy())
        q.put(res)
    except Exception as e:                      # reported to the parent
        q.put(repr(e))


def test_checked_build_finds_no_index_error(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_worker, args=(q,))
    p.start()
    try:
        res = q.get(timeout=600)
    finally:
        p.join(timeout=120)
        if p.is_alive():
            p.kill()
            p.join()
    assert not isinstance(res, str), res
    batches = _batches()
    for name, bn, call, k, K, form, slots in _cases():
        rc, got = res[name]
        assert rc == 0, f"{name}: status {rc}"
        b = batches[bn]
        if call in ("sketch", "noalloc"):
            exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 7, threads=THREADS)
            assert np.array_equal(got.view(np.uint64).reshape(exp.shape), exp), name
        elif call == "lsh":
            exp = oracle_mod.lsh(b.indptr, b.indices, b.weights, k, K, 7, threads=THREADS)
            assert np.array_equal(got.view(np.uint32).reshape(exp.shape), exp), name
        else:
            exp = oracle_mod.bottomk(b.indptr, b.indices, b.weights, k, 7, threads=THREADS)
            assert np.array_equal(got.view(np.uint64).reshape(exp.shape), exp), name
