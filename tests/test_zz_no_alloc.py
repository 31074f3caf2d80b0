"""dm_sketch_noalloc, the entry point for host programs that do not let a library allocate device
memory (for example a framework whose caching allocator owns the whole device).  Called through
the C ABI, it must give exactly the oracle's keys (and so dm_sketch's), on two calls in a row:
the shared scratch keeps the previous call's contents, so the second call checks that the
library clears what must start at zero.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

THREADS = 16


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


def _noalloc(torch, lib, b, k, seed, stream=None):
    ip, ix, w = _dev(torch, b)
    out = torch.full((b.n_sets, k), -1, dtype=torch.int64, device="cuda")
    P = ctypes.c_void_p
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.dm_sketch_noalloc(P(ip.data_ptr()), P(ix.data_ptr()), P(w.data_ptr()), b.n_sets, k, seed,
                               P(out.data_ptr()), P(st.cuda_stream))
    return rc, out.cpu().numpy().view(np.uint64)


def test_noalloc_matches_oracle_twice(env, oracle_mod):
    torch, dmx, lib = env
    # both kernels: norms from 1e-3 (general walk) to 1e3 (fast walk), ragged rows, empty rows
    first = workloads.random_sets(3000, 0, 300, 1 << 24, seed=501)
    second = workloads.workload0(700)
    rc, got = _noalloc(torch, lib, first, 256, 7)
    assert rc == 0
    assert np.array_equal(got, oracle_mod.sketch(first.indptr, first.indices, first.weights, 256, 7, threads=THREADS))
    rc, got = _noalloc(torch, lib, second, 64, 1)
    assert rc == 0
    assert np.array_equal(got, oracle_mod.sketch(second.indptr, second.indices, second.weights, 64, 1,
                                                 threads=THREADS))


@pytest.mark.parametrize("k,n", [(1024, 400), (8192, 40)])
def test_noalloc_large_k(env, oracle_mod, k, n):
    """Bucket counts whose shared memory leaves room for one or two warps per block (the launch
    shape the call picks for itself), against the oracle and against dm_sketch."""
    torch, dmx, lib = env
    b = workloads.random_sets(n, 0, 300, 1 << 24, seed=503 + k)
    rc, got = _noalloc(torch, lib, b, k, 11)
    assert rc == 0
    assert np.array_equal(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 11, threads=THREADS))
    ctx = dmx.dm_create(0)
    ref = dmx.dm_sketch(ctx, *_dev(torch, b), k, 11)
    dmx.dm_sync_status(ctx)
    ctx.close()
    assert np.array_equal(got, ref.cpu().numpy().view(np.uint64))


def test_noalloc_python_wrapper(env, oracle_mod):
    torch, dmx, lib = env
    b = workloads.workload0(300)
    ip, ix, w = _dev(torch, b)
    out = torch.empty((b.n_sets, 64), dtype=torch.int64, device="cuda")
    dmx.dm_sketch_noalloc(ip, ix, w, 64, 1, out)
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1, threads=THREADS)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), exp)
    with pytest.raises(ValueError):
        dmx.dm_sketch_noalloc(ip, ix, w, 64, 1, out[:-1])              # one row short
    with pytest.raises(TypeError):
        dmx.dm_sketch_noalloc(ip, ix, w, 64, 1, out.cpu())             # host memory


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")     # the refused call captures nothing
def test_noalloc_refuses_a_capturing_stream(env):
    torch, dmx, lib = env
    b = workloads.workload0(50)
    ip, ix, w = _dev(torch, b)
    out = torch.empty((b.n_sets, 64), dtype=torch.int64, device="cuda")
    P = ctypes.c_void_p
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    rcs = []
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            rcs.append(lib.dm_sketch_noalloc(P(ip.data_ptr()), P(ix.data_ptr()), P(w.data_ptr()), b.n_sets, 64, 1,
                                             P(out.data_ptr()), P(st.cuda_stream)))
    assert rcs == [1]                                  # DM_EINVAL: the call would synchronise the stream
    rc, got = _noalloc(torch, lib, b, 64, 1)            # the next call works as usual
    assert rc == 0


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
