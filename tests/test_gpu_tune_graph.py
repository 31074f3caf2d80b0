"""GPU tests of the launch machinery around the kernels: CUDA-graph replay (DM_OPT_GRAPH) and the
launch-setting search (dm_autotune).  Neither may change a bit: every output is compared with the
oracle or with the plain launch of the same call."""
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


def keys(out):
    return out.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def heavy():
    """Heavy-tailed rows (log-normal nnz, median 100, sigma 1.5, up to 20,000; ||x||_1 over six
    decades): exercises every class of the batched form."""
    return workloads.workload2(1500)


@pytest.mark.parametrize("form", [0, 1, 2])
def test_graph_replay_matches_oracle(dmx, torch_mod, oracle_mod, heavy, form):
    torch = torch_mod
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_FORM, form)
    dmx.dm_set_option(ctx, dmx.OPT_LARGE_NNZ, 1000)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    ip, ix, w = to_dev(torch, heavy)
    k = 256
    exp = oracle_mod.sketch(heavy.indptr, heavy.indices, heavy.weights, k, 5, threads=THREADS)
    out = torch.empty(heavy.n_sets * k, dtype=torch.int64, device="cuda")
    for rep in range(3):                      # capture, then two replays of the cached graph
        out.fill_(0)
        dmx.dm_sketch(ctx, ip, ix, w, k, 5, out=out)
        assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
        assert np.array_equal(keys(out).reshape(-1, k), exp), f"form {form} call {rep}"
    ctx.close()


def test_graph_update_and_cache(dmx, torch_mod, oracle_mod):
    """New seeds, sizes, outputs and kinds: each call is a new plan, patched into a cached
    executable of the same shape or captured anew (more plans than the cache holds)."""
    torch = torch_mod
    ctx = dmx.dm_create(0)
    ref = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    b = workloads.random_sets(700, 0, 400, 1 << 24, seed=91)
    ip, ix, w = to_dev(torch, b)
    for i in range(20):
        seed = 1000 + i
        k = (64, 100, 256)[i % 3]
        n = 700 - 13 * i
        sub_ip = ip[: n + 1]
        got = dmx.dm_sketch(ctx, sub_ip, ix, w, k, seed)
        exp = dmx.dm_sketch(ref, sub_ip, ix, w, k, seed)
        assert np.array_equal(keys(got), keys(exp)), f"call {i}"
        if i % 5 == 0:
            words = dmx.dm_sketch_bbit(ctx, sub_ip, ix, w, k, 1, seed)
            words_ref = dmx.dm_sketch_bbit(ref, sub_ip, ix, w, k, 1, seed)
            assert np.array_equal(keys(words), keys(words_ref))
            lg = dmx.dm_lsh(ctx, sub_ip, ix, w, 16, 4, seed)
            lr = dmx.dm_lsh(ref, sub_ip, ix, w, 16, 4, seed)
            assert torch.equal(lg, lr)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    # spot check against the oracle after many updates
    got = dmx.dm_sketch(ctx, ip, ix, w, 256, 77)
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, 256, 77, threads=THREADS)
    assert np.array_equal(keys(got).reshape(-1, 256), exp)
    # turning replay off drops the cache and keeps the bits
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 0)
    again = dmx.dm_sketch(ctx, ip, ix, w, 256, 77)
    assert torch.equal(again, got)
    ctx.close()
    ref.close()


def test_graph_reports_kernel_errors(dmx, torch_mod):
    """A bad weight is still reported by the graph-launched kernels, on every replay."""
    torch = torch_mod
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_GRAPH, 1)
    b = workloads.csr_of([(np.array([1, 2], np.uint32), np.array([0.5, -1.0], np.float32)),
                          (np.array([3], np.uint32), np.array([0.25], np.float32))])
    ip, ix, w = to_dev(torch, b)
    for _ in range(2):
        out = dmx.dm_sketch(ctx, ip, ix, w, 64, 1)
        assert dmx.dm_sync_status(ctx, raise_on_error=False) == 1
        k = keys(out).reshape(2, 64)
        assert np.all(k[0] == np.uint64(2 ** 64 - 1))
        assert np.all(k[1] != np.uint64(2 ** 64 - 1))
    ctx.close()


def test_autotune_keeps_bits_sketch(dmx, torch_mod, oracle_mod, heavy):
    torch = torch_mod
    ctx = dmx.dm_create(0)
    ip, ix, w = to_dev(torch, heavy)
    k = 1024
    before = dmx.dm_sketch(ctx, ip, ix, w, k, 3)
    res = dmx.dm_autotune(ctx, ip, ix, w, k, 3, max_sets=1000)
    assert res["form"] in (0, 2)
    assert 1 <= res["warps_per_block"] <= 8
    assert res["phi0_1024"] in (1024, 1280, 1536, 2048)
    assert res["sets_timed"] == 1000
    assert res["slots"] in (0, 1, 2)
    assert 0 < res["ms_tuned"] <= res["ms_default"]
    after = dmx.dm_sketch(ctx, ip, ix, w, k, 3)
    assert torch.equal(before, after)
    exp = oracle_mod.sketch(heavy.indptr, heavy.indices, heavy.weights, k, 3, threads=THREADS)
    assert np.array_equal(keys(after).reshape(-1, k), exp)
    # b-bit calls are a different kind: tuned separately, same words either way
    wb = dmx.dm_sketch_bbit(ctx, ip, ix, w, 64, 1, 9)
    dmx.dm_autotune(ctx, ip, ix, w, 64, 9, b=1)
    assert torch.equal(dmx.dm_sketch_bbit(ctx, ip, ix, w, 64, 1, 9), wb)
    # ignoring and forgetting the stored choice
    dmx.dm_set_option(ctx, dmx.OPT_TUNED, 0)
    assert torch.equal(dmx.dm_sketch(ctx, ip, ix, w, k, 3), before)
    dmx.dm_set_option(ctx, dmx.OPT_TUNED, 1)
    dmx.dm_set_option(ctx, dmx.OPT_TUNED, 2)
    assert torch.equal(dmx.dm_sketch(ctx, ip, ix, w, k, 3), before)
    ctx.close()


def test_autotune_keeps_bits_lsh(dmx, torch_mod, oracle_mod):
    torch = torch_mod
    ctx = dmx.dm_create(0)
    b = workloads.random_sets(600, 1, 300, 1 << 20, seed=44)
    ip, ix, w = to_dev(torch, b)
    before = dmx.dm_lsh(ctx, ip, ix, w, 32, 4, 8)
    res = dmx.dm_autotune(ctx, ip, ix, w, 32, 8, lsh_K=4)
    assert res["phi0_1024"] in (2048, 3072, 4096, 6144, 8192)
    after = dmx.dm_lsh(ctx, ip, ix, w, 32, 4, 8)
    assert torch.equal(before, after)
    exp = oracle_mod.lsh(b.indptr, b.indices, b.weights, 32, 4, 8, threads=THREADS)
    assert np.array_equal(after.cpu().numpy().view(np.uint32).reshape(-1, 32), exp)
    ctx.close()


def test_autotune_rejects_bad_arguments(dmx, torch_mod):
    torch = torch_mod
    ctx = dmx.dm_create(0)
    b = workloads.random_sets(10, 1, 10, 1000, seed=2)
    ip, ix, w = to_dev(torch, b)
    for kw in ({"k": 0}, {"k": 64, "b": 3}, {"k": 2000, "lsh_K": 4}):
        with pytest.raises(dmx.DartMinHashError):
            dmx.dm_autotune(ctx, ip, ix, w, kw.pop("k"), 1, **kw)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_autotune(ctx, ip[:1], ix, w, 64, 1)          # no rows
    ctx.close()


def test_saved_tunings_reinstall(dmx, torch_mod, tmp_path):
    """Settings chosen by dm_autotune, saved to JSON and installed into a fresh context, change no
    bit of its calls; settings outside the options' ranges are rejected."""
    torch = torch_mod
    b = workloads.random_sets(3000, 1, 300, 1 << 24, seed=23)
    ip, ix, w = to_dev(torch, b)
    c1 = dmx.dm_create(0)
    t = dmx.dm_autotune(c1, ip, ix, w, 256, 9, max_sets=3000)
    ref = dmx.dm_sketch(c1, ip, ix, w, 256, 9)
    path = str(tmp_path / "tunings.json")
    dmx.save_tunings(path, [{"k": 256, "b": 0, "tuning": t}])
    c2 = dmx.dm_create(0)
    assert dmx.load_tunings(c2, path) == 1
    assert torch.equal(dmx.dm_sketch(c2, ip, ix, w, 256, 9), ref)
    bad = dict(t, form=7)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_set_tuning(c2, 256, bad)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_set_tuning(c2, 256, dict(t, slots=3))
    # the other slot layout, installed as a tuning, gives the same bits
    dmx.dm_set_tuning(c2, 256, dict(t, slots=2 if t["slots"] != 2 else 1))
    assert torch.equal(dmx.dm_sketch(c2, ip, ix, w, 256, 9), ref)
    assert dmx.dm_sync_status(c2, raise_on_error=False) == 0
    c1.close()
    c2.close()
