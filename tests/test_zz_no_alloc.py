"""dm_sketch_noalloc, the entry point for host programs that do not let a library allocate
device memory (for example a framework whose caching allocator owns the whole device).  It is
called through the C ABI and must give exactly the keys of dm_sketch, on two calls in a row (the
shared scratch keeps the previous call's contents, so the second call checks that the library
clears what must start at zero).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    return torch, dmx, dmx.load()


def _dev(torch, b):
    return (torch.from_numpy(np.ascontiguousarray(b.indptr, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.indices, dtype=np.uint32).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.weights, dtype=np.float32)).cuda())


def _noalloc(torch, lib, b, k, seed):
    ip, ix, w = _dev(torch, b)
    out = torch.full((b.n_sets, k), -1, dtype=torch.int64, device="cuda")
    P = ctypes.c_void_p
    rc = lib.dm_sketch_noalloc(P(ip.data_ptr()), P(ix.data_ptr()), P(w.data_ptr()), b.n_sets, k, seed,
                               P(out.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    return rc, out.cpu().numpy().view(np.uint64)


def _reference(torch, dmx, b, k, seed):
    ctx = dmx.dm_create(0)
    ip, ix, w = _dev(torch, b)
    out = dmx.dm_sketch(ctx, ip, ix, w, k, seed)
    dmx.dm_sync_status(ctx)
    ctx.close()
    return out.cpu().numpy().view(np.uint64)


def test_noalloc_matches_dm_sketch_twice(env):
    torch, dmx, lib = env
    # both kernels: norms from 1e-3 (general walk) to 1e3 (fast walk), ragged rows, empty rows
    first = workloads.random_sets(3000, 0, 300, 1 << 24, seed=501)
    second = workloads.workload0(700)
    rc, got = _noalloc(torch, lib, first, 256, 7)
    assert rc == 0
    assert np.array_equal(got, _reference(torch, dmx, first, 256, 7))
    rc, got = _noalloc(torch, lib, second, 64, 1)
    assert rc == 0
    assert np.array_equal(got, _reference(torch, dmx, second, 64, 1))


def test_noalloc_rejects_oversized_batches(env):
    torch, dmx, lib = env
    n = dmx.NOALLOC_MAX_SETS + 1
    P = ctypes.c_void_p
    ip = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    out = torch.empty((n, 1), dtype=torch.int64, device="cuda")
    rc = lib.dm_sketch_noalloc(P(ip.data_ptr()), P(ip.data_ptr()), P(ip.data_ptr()), n, 1, 1,
                               P(out.data_ptr()), P(torch.cuda.current_stream().cuda_stream))
    assert rc == 1                                 # DM_EINVAL, before any GPU work


def test_noalloc_reports_bad_weights(env):
    torch, dmx, lib = env
    b = workloads.csr_of([(np.array([1, 2], np.uint32), np.array([0.5, -1.0], np.float32)),
                          (np.array([3], np.uint32), np.array([0.25], np.float32))])
    rc, got = _noalloc(torch, lib, b, 32, 3)
    assert rc == 1 and (got[0] == np.uint64(2 ** 64 - 1)).all()
    rc, got = _noalloc(torch, lib, b.rows([1]), 32, 3)   # the status does not leak into the next call
    assert rc == 0
