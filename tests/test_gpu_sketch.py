"""GPU parity of dm_sketch / dm_sketch_bbit with the oracle: bit-exact uint64 keys (integer
work, so the bar is exact equality), at small sizes in full and at the full W1/W2 sizes on
sampled rows, in the launch configuration the bench uses, plus edge cases."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

U64MAX = np.uint64(2 ** 64 - 1)
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


def to_dev(torch, b):
    return (torch.from_numpy(np.ascontiguousarray(b.indptr, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.indices, dtype=np.uint32).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(b.weights, dtype=np.float32)).cuda())


def gpu_sketch(dmx, torch, ctx, b, k, seed):
    ip, ix, w = to_dev(torch, b)
    out = dmx.dm_sketch(ctx, ip, ix, w, k, seed)
    rc = dmx.dm_sync_status(ctx, raise_on_error=False)
    return out.cpu().numpy().view(np.uint64), rc


def assert_same(got, exp, what=""):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        r, c = bad[0]
        raise AssertionError(f"{what}: {len(bad)} mismatches; first row {r} slot {c}: "
                             f"gpu {int(got[r, c]):016x} oracle {int(exp[r, c]):016x}")


def test_w0_full_parity(dmx, torch_mod, ctx, oracle_mod):
    """W0 in full: 1,000 sets, 64 elements, k = 64, seed 1."""
    b = workloads.workload0()
    got, rc = gpu_sketch(dmx, torch_mod, ctx, b, 64, 1)
    assert rc == 0
    assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1, threads=THREADS), "W0")


@pytest.mark.parametrize("k", [1, 2, 7, 64, 100, 256, 1000, 1024])
def test_ragged_sets_parity(dmx, torch_mod, ctx, oracle_mod, k):
    """Ragged nnz (0..300, several 32-element tiles and a ragged tail), ||x||_1 over six
    decades, several k including non powers of two."""
    b = workloads.random_sets(300, 0, 300, 1 << 24, seed=10 + k)
    got, rc = gpu_sketch(dmx, torch_mod, ctx, b, k, 12345)
    assert rc == 0
    assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 12345, threads=THREADS), f"k={k}")


@pytest.mark.parametrize("form", [0, 1, 2])
def test_largest_k_parity(dmx, torch_mod, oracle_mod, form):
    """The largest bucket counts the library takes (k up to 8,192: 64 KB of buckets per set),
    keys and 1-bit words, in every launch form."""
    b = workloads.random_sets(40, 0, 300, 1 << 24, seed=77)
    c = dmx.dm_create(0)
    dmx.dm_set_option(c, dmx.OPT_FORM, form)
    ip, ix, w = to_dev(torch_mod, b)
    for k in (4097, 8192):
        got, rc = gpu_sketch(dmx, torch_mod, c, b, k, 4242)
        assert rc == 0
        exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 4242, threads=THREADS)
        assert_same(got, exp, f"k={k} form={form}")
    words = dmx.dm_sketch_bbit(c, ip, ix, w, 8192, 1, 4242)
    assert dmx.dm_sync_status(c, raise_on_error=False) == 0
    ew = oracle_mod.sketch_bbit(b.indptr, b.indices, b.weights, 8192, 1, 4242, threads=THREADS)
    assert np.array_equal(words.cpu().numpy().view(np.uint64), ew)
    c.close()


def test_extreme_norms_parity(dmx, torch_mod, ctx, oracle_mod):
    """||x||_1 from 1e-6 to 1e6: many rank regions (small norms) or many weight regions."""
    rows = []
    rng = np.random.default_rng(3)
    for l1 in [1e-6, 1e-4, 1e-2, 1.0, 1e2, 1e4, 1e6]:
        for nnz in [1, 5, 40]:
            idx = np.sort(rng.choice(1 << 30, nnz, replace=False)).astype(np.uint32)
            z = rng.exponential(size=nnz)
            rows.append((idx, (z / z.sum() * l1).astype(np.float32)))
    b = workloads.csr_of(rows)
    for k in (16, 256):
        got, rc = gpu_sketch(dmx, torch_mod, ctx, b, k, 99)
        assert rc == 0
        assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 99), f"k={k}")


def test_large_weights_parity(dmx, torch_mod, ctx, oracle_mod):
    """Weights with t x_i >= 2^31 (weight regions above 31, handled by the general kernel)
    beside ordinary rows, up to the 2^39 limit."""
    rng = np.random.default_rng(12)
    rows = []
    for big in [1e7, 1e8, 3e8]:
        for nnz in [1, 3, 33]:
            idx = np.sort(rng.choice(1 << 30, nnz, replace=False)).astype(np.uint32)
            w = rng.exponential(size=nnz).astype(np.float32)
            w[0] = np.float32(big)
            rows.append((idx, w))
        rows.append((np.array([5, 6], np.uint32), np.array([0.5, 2.0], np.float32)))
    b = workloads.csr_of(rows)
    for k in (64, 256):
        got, rc = gpu_sketch(dmx, torch_mod, ctx, b, k, 31)
        assert rc == 0
        assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 31), f"k={k}")


def test_edge_cases_parity(dmx, torch_mod, ctx, oracle_mod):
    f = np.float32
    rows = [
        ([], []),                                         # empty row
        ([3, 4], [0.0, 0.0]),                             # all zero -> sentinel
        ([7], [1.0]),                                     # single element
        ([1, 2, 3], [0.0, 0.5, 0.0]),                     # zeros inside
        ([5, 5, 5], [0.25, 0.75, 0.5]),                   # duplicates act as the max
        ([5], [0.75]),
        ([0, 4294967295], [1e-30, 2.5]),                  # extreme index and tiny weight
        ([11, 12], [np.float32(1e-40), 0.5]),             # subnormal weight beside a normal one
        ([9, 10], [-0.0, 3.0]),                           # negative zero is a zero weight
    ]
    # weights whose t x lands exactly on a region edge 2^nu - 1 for k = 2 (t = 4)
    rows += [([20, 21], [0.75, 1.75]), ([22], [0.25])]
    b = workloads.csr_of([(np.array(i, np.uint32), np.array(w, f)) for i, w in rows])
    for k in (1, 2, 3, 64):
        got, rc = gpu_sketch(dmx, torch_mod, ctx, b, k, 5)
        assert rc == 0
        exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 5)
        assert_same(got, exp, f"k={k}")
    assert (got[0] == U64MAX).all() and (got[1] == U64MAX).all()
    assert (got[4] == got[5]).all()


def test_large_row_parity(dmx, torch_mod, ctx, oracle_mod):
    """One set with 100,000 elements (the W2 clip) next to tiny ones."""
    rng = np.random.default_rng(44)
    big = np.sort(rng.choice(1 << 24, 100_000, replace=False)).astype(np.uint32)
    rows = [(big, rng.lognormal(size=100_000).astype(np.float32)),
            (np.array([1], np.uint32), np.array([0.5], np.float32))]
    b = workloads.csr_of(rows)
    got, rc = gpu_sketch(dmx, torch_mod, ctx, b, 1024, 8)
    assert rc == 0
    assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, 1024, 8), "big")


def test_invalid_and_out_of_range_weights(dmx, torch_mod, ctx, oracle_mod):
    f = np.float32
    rows = [([1, 2], [0.5, 0.5]), ([1, 2], [0.5, -1.0]), ([3], [np.nan]), ([4], [np.inf]),
            ([5, 6], [0.25, 0.125])]
    b = workloads.csr_of([(np.array(i, np.uint32), np.array(w, f)) for i, w in rows])
    got, rc = gpu_sketch(dmx, torch_mod, ctx, b, 32, 3)
    assert rc == 1                                              # DM_EINVAL
    assert (got[1:4] == U64MAX).all()
    good = b.rows([0, 4])
    assert_same(got[[0, 4]], oracle_mod.sketch(good.indptr, good.indices, good.weights, 32, 3), "valid rows")
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0   # status cleared
    # a weight with t x >= 2^39 - 1, and a set whose only weight is subnormal (it would need
    # a rank limit near 1e40): both outside the supported range on both sides
    for bad_w in [2.0 ** 39, 1e-40]:
        big = workloads.csr_of([(np.array([1], np.uint32), np.array([bad_w], f))])
        got, rc = gpu_sketch(dmx, torch_mod, ctx, big, 1, 3)
        assert rc == 5                                          # DM_ERANGE
        assert (got == U64MAX).all()
        with pytest.raises(oracle_mod.OracleError) as e:
            oracle_mod.sketch(big.indptr, big.indices, big.weights, 1, 3)
        assert e.value.code == 5


def test_misaligned_arrays_are_rejected(dmx, torch_mod, ctx):
    """An array not aligned to its element size is refused before any launch (DM_EINVAL); the
    weights of aligned rows at every offset mod 4 (the 128-bit row scans' ragged ends) are
    covered by the ragged-set tests."""
    torch = torch_mod
    b = workloads.random_sets(10, 1, 20, 1000, seed=3)
    ip, ix, w = to_dev(torch, b)
    out = torch.empty((10, 64), dtype=torch.int64, device="cuda")
    lib = dmx.load()
    cases = ((ip.data_ptr() + 4, ix.data_ptr(), w.data_ptr()), (ip.data_ptr(), ix.data_ptr() + 2, w.data_ptr()),
             (ip.data_ptr(), ix.data_ptr(), w.data_ptr() + 1))
    for dip, dix, dw in cases:
        rc = lib.dm_sketch(ctx.handle, ctypes_ptr(dip), ctypes_ptr(dix), ctypes_ptr(dw), 10, 64, 1,
                           ctypes_ptr(out.data_ptr()), dmx._stream(None))
        assert rc == 1
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0


def ctypes_ptr(v):
    import ctypes
    return ctypes.c_void_p(v)


@pytest.mark.parametrize("bits", [1, 2, 4, 8, 16, 32])
def test_bbit_parity(dmx, torch_mod, ctx, oracle_mod, bits):
    b = workloads.random_sets(200, 1, 120, 1 << 20, seed=70 + bits)
    ip, ix, w = to_dev(torch_mod, b)
    for k in (64, 100, 256):
        keys = torch_mod.empty((b.n_sets, k), dtype=torch_mod.int64, device="cuda")
        words = dmx.dm_sketch_bbit(ctx, ip, ix, w, k, bits, 21, out_keys=keys)
        assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
        ew, ek = oracle_mod.sketch_bbit(b.indptr, b.indices, b.weights, k, bits, 21, keys=True,
                                        threads=THREADS)
        assert_same(words.cpu().numpy().view(np.uint64), ew, f"b={bits} k={k} words")
        assert_same(keys.cpu().numpy().view(np.uint64), ek, f"b={bits} k={k} keys")


def test_options_do_not_change_bits(dmx, torch_mod, ctx):
    b = workloads.random_sets(400, 1, 200, 1 << 24, seed=5)
    ref, _ = gpu_sketch(dmx, torch_mod, ctx, b, 256, 77)
    again, _ = gpu_sketch(dmx, torch_mod, ctx, b, 256, 77)
    assert_same(again, ref, "repeat")
    for opt, val in [(dmx.OPT_PHI0, 512), (dmx.OPT_PHI0, 4096), (dmx.OPT_PHI0, 1024 * 3),
                     (dmx.OPT_WARPS_PER_BLOCK, 1), (dmx.OPT_WARPS_PER_BLOCK, 3),
                     (dmx.OPT_FORM, dmx.FORM_PLAIN), (dmx.OPT_FORM, dmx.FORM_PERSISTENT),
                     (dmx.OPT_LARGE_NNZ, 0), (dmx.OPT_LARGE_NNZ, 40), (dmx.OPT_LARGE_NNZ, 150),
                     (dmx.OPT_SLOTS, dmx.SLOTS_SHARED), (dmx.OPT_SLOTS, dmx.SLOTS_ROW)]:
        c2 = dmx.dm_create(0)
        dmx.dm_set_option(c2, opt, val)
        got, rc = gpu_sketch(dmx, torch_mod, c2, b, 256, 77)
        c2.close()
        assert rc == 0
        assert_same(got, ref, f"option {opt}={val}")


@pytest.mark.parametrize("form", [0, 1, 2])
def test_forms_on_heavy_tailed_batch(dmx, torch_mod, oracle_mod, form):
    """Batched (large sets on blocks of 8 warps, largest first), plain and persistent forms on a
    heavy-tailed batch: same bits as the oracle."""
    rng = np.random.default_rng(66)
    rows = []
    for s in range(400):
        nnz = int(min(20000, max(1, np.exp(np.log(60) + 1.5 * rng.standard_normal()))))
        idx = np.sort(rng.choice(1 << 24, nnz, replace=False)).astype(np.uint32)
        z = rng.lognormal(size=nnz)
        rows.append((idx, (z / z.sum() * 10 ** rng.uniform(-3, 3)).astype(np.float32)))
    b = workloads.csr_of(rows)
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_FORM, form)
    dmx.dm_set_option(c2, dmx.OPT_LARGE_NNZ, 500)
    for k in (64, 1024):
        got, rc = gpu_sketch(dmx, torch_mod, c2, b, k, 17)
        assert rc == 0
        assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 17, threads=THREADS), f"form {form} k={k}")
    c2.close()


@pytest.mark.parametrize("slots", [1, 2])
@pytest.mark.parametrize("form", [0, 1, 2])
def test_slot_storage_layouts(dmx, torch_mod, oracle_mod, form, slots):
    """Bucket minima in shared memory (1) or in the output row with shared rank codes as a filter
    (2), at small and large k, in every form (the batched one with a block-per-set class): the
    oracle's bits either way."""
    rng = np.random.default_rng(91)
    rows = []
    for s in range(300):
        nnz = int(min(5000, max(1, np.exp(np.log(60) + 1.3 * rng.standard_normal()))))
        idx = np.sort(rng.choice(1 << 24, nnz, replace=False)).astype(np.uint32)
        z = rng.lognormal(size=nnz)
        rows.append((idx, (z / z.sum() * 10 ** rng.uniform(-3, 3)).astype(np.float32)))
    b = workloads.csr_of(rows)
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_FORM, form)
    dmx.dm_set_option(c2, dmx.OPT_SLOTS, slots)
    dmx.dm_set_option(c2, dmx.OPT_LARGE_NNZ, 400)
    for k in (7, 256, 1024):
        got, rc = gpu_sketch(dmx, torch_mod, c2, b, k, 29)
        assert rc == 0
        assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 29, threads=THREADS),
                    f"form {form} slots {slots} k={k}")
    c2.close()


@pytest.mark.parametrize("k", [1, 64, 1024])
def test_block_per_set_split_and_stride(dmx, torch_mod, oracle_mod, k):
    """Every non-empty set on a block of 8 warps (large-set threshold 1): sets below 512 elements
    split each tile's areas among the warps, larger ones deal their tiles; norms over six
    decades exercise both walks."""
    rng = np.random.default_rng(70 + k)
    rows = []
    for s in range(160):
        nnz = int(rng.choice([0, 1, 2, 5, 31, 33, 100, 511, 512, 700, 3000]))
        idx = np.sort(rng.choice(1 << 24, nnz, replace=False)).astype(np.uint32)
        z = rng.lognormal(size=nnz)
        rows.append((idx, (z / max(z.sum(), 1e-30) * 10 ** rng.uniform(-3, 3)).astype(np.float32)))
    b = workloads.csr_of(rows)
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_LARGE_NNZ, 1)
    got, rc = gpu_sketch(dmx, torch_mod, c2, b, k, 23)
    c2.close()
    assert rc == 0
    assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 23, threads=THREADS), f"k={k}")


def test_large_class_by_work_estimate(dmx, torch_mod, oracle_mod):
    """Sets sent to the block kernel by their work estimate (DM_OPT_LARGE_WORK) rather than their
    size: same bits as the oracle."""
    b = workloads.workload2(600)
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_LARGE_NNZ, 0)
    dmx.dm_set_option(c2, dmx.OPT_LARGE_WORK, 12000)
    for k in (64, 1024):
        got, rc = gpu_sketch(dmx, torch_mod, c2, b, k, 29)
        assert rc == 0
        assert_same(got, oracle_mod.sketch(b.indptr, b.indices, b.weights, k, 29, threads=THREADS), f"k={k}")
    c2.close()


def test_counters_and_streams(dmx, torch_mod, ctx, oracle_mod):
    torch = torch_mod
    b = workloads.workload0(300)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    c2 = dmx.dm_create(0)
    dmx.dm_set_option(c2, dmx.OPT_COUNTERS, cnt.data_ptr())
    dmx.dm_set_option(c2, dmx.OPT_PHI0, 1024)             # phi0 = 1, as the oracle below
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ip, ix, w = to_dev(torch, b)
        out = dmx.dm_sketch(c2, ip, ix, w, 64, 1, stream=s)
    assert dmx.dm_sync_status(c2, stream=s, raise_on_error=False) == 0
    c2.close()
    got = out.cpu().numpy().view(np.uint64)
    exp, wk = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1, work=True)
    assert_same(got, exp, "counted")
    areas, darts, kept, passes = cnt.cpu().tolist()
    assert abs(passes - wk[:, 3].sum()) <= 2              # same retry decisions as the oracle
    assert abs(darts - areas) < 5 * areas ** 0.5          # Poi(1) darts per area
    assert kept >= wk[:, 2].sum() * 0.5


@pytest.mark.parametrize("mode", ["staged", "in_place", "auto"])
def test_host_entry_matches_device(dmx, torch_mod, oracle_mod, mode):
    """dm_sketch_host in each way of moving the data (staged chunked copies; kernels reading and
    writing the page-locked host arrays in place; the automatic choice): keys and 1-bit words
    equal the device entry's and the oracle's."""
    torch = torch_mod
    ctx = dmx.dm_create(0)
    dmx.dm_set_option(ctx, dmx.OPT_HOST_MODE, {"staged": dmx.HOST_STAGED, "in_place": dmx.HOST_IN_PLACE,
                                               "auto": dmx.HOST_AUTO}[mode])
    b = workloads.random_sets(500, 1, 100, 1 << 20, seed=8)
    ref, _ = gpu_sketch(dmx, torch, ctx, b, 128, 4)
    assert_same(ref, oracle_mod.sketch(b.indptr, b.indices, b.weights, 128, 4, threads=THREADS), "device entry")
    ip = torch.from_numpy(b.indptr.astype(np.int64)).pin_memory()
    ix = torch.from_numpy(b.indices.view(np.int32)).pin_memory()
    w = torch.from_numpy(b.weights).pin_memory()
    out = torch.empty((b.n_sets, 128), dtype=torch.int64).pin_memory()
    dmx.dm_sketch_host(ctx, ip, ix, w, 128, 4, out)
    assert_same(out.numpy().view(np.uint64), ref, "host entry")
    # keys and 1-bit words together, batch split into several chunks when staged
    big = workloads.random_sets(40_000, 1, 64, 1 << 20, seed=9)
    ref2, _ = gpu_sketch(dmx, torch, ctx, big, 64, 6)
    ipb = torch.from_numpy(big.indptr.astype(np.int64)).pin_memory()
    ixb = torch.from_numpy(big.indices.view(np.int32)).pin_memory()
    wb = torch.from_numpy(big.weights).pin_memory()
    kh, wh = dmx.dm_sketch_host(ctx, ipb, ixb, wb, 64, 6,
                                out_keys=torch.empty((big.n_sets, 64), dtype=torch.int64).pin_memory(),
                                out_words=torch.empty((big.n_sets, 1), dtype=torch.int64).pin_memory(), b=1)
    assert_same(kh.numpy().view(np.uint64), ref2, "host entry keys")
    dev_words = dmx.dm_sketch_bbit(ctx, *to_dev(torch, big), 64, 1, 6)
    assert_same(wh.numpy().view(np.uint64), dev_words.cpu().numpy().view(np.uint64), "host entry words")
    # an output in ordinary (not page-locked) memory: staged and automatic modes copy, in place refuses
    plain = torch.empty((b.n_sets, 128), dtype=torch.int64)
    if mode == "in_place":
        with pytest.raises(dmx.DartMinHashError) as e:
            dmx.dm_sketch_host(ctx, ip, ix, w, 128, 4, plain)
        assert e.value.code == 1
    else:
        dmx.dm_sketch_host(ctx, ip, ix, w, 128, 4, plain)
        assert_same(plain.numpy().view(np.uint64), ref, "host entry, pageable output")
    ctx.close()


@pytest.fixture(scope="module")
def w1():
    return workloads.workload1()


def test_w1_full_size_sampled(dmx, torch_mod, ctx, oracle_mod, w1):
    """W1 at full size (1,000,000 sets, k = 256, keys and 1-bit words in one call, as the
    bench runs it); 3,000 rows spread over the batch checked against the oracle."""
    torch = torch_mod
    ip, ix, w = to_dev(torch, w1)
    keys = torch.empty((w1.n_sets, 256), dtype=torch.int64, device="cuda")
    words = dmx.dm_sketch_bbit(ctx, ip, ix, w, 256, 1, 1, out_keys=keys)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    rng = np.random.default_rng(0)
    sel = np.unique(np.concatenate([rng.choice(w1.n_sets, 2990, replace=False),
                                    np.arange(5), np.arange(w1.n_sets - 5, w1.n_sets)]))
    sub = w1.rows(sel)
    ew, ek = oracle_mod.sketch_bbit(sub.indptr, sub.indices, sub.weights, 256, 1, 1, keys=True,
                                    threads=THREADS)
    sel_t = torch.from_numpy(sel).cuda()
    assert_same(keys[sel_t].cpu().numpy().view(np.uint64), ek, "W1 keys")
    assert_same(words[sel_t].cpu().numpy().view(np.uint64), ew, "W1 1-bit")
    assert (keys.cpu().numpy().view(np.uint64) != U64MAX).all()


def test_w2_full_size_sampled(dmx, torch_mod, ctx, oracle_mod):
    """W2 at full size (200,000 heavy-tailed sets, k = 1024); sampled rows, plus the ten
    largest sets."""
    torch = torch_mod
    b = workloads.workload2()
    ip, ix, w = to_dev(torch, b)
    out = dmx.dm_sketch(ctx, ip, ix, w, 1024, 1)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    lens = np.diff(b.indptr)
    rng = np.random.default_rng(1)
    sel = np.unique(np.concatenate([rng.choice(b.n_sets, 600, replace=False), np.argsort(lens)[-10:]]))
    sub = b.rows(sel)
    exp = oracle_mod.sketch(sub.indptr, sub.indices, sub.weights, 1024, 1, threads=THREADS)
    assert_same(out[torch.from_numpy(sel).cuda()].cpu().numpy().view(np.uint64), exp, "W2")


def test_row_range_shards_on_streams_match_whole_batch(dmx, torch_mod, ctx):
    """What N ranks do (each sketches its own contiguous rows): three row-range shards, each
    on its own context and stream, launched together, give the bits of one whole-batch call."""
    torch = torch_mod
    b = workloads.random_sets(3000, 0, 300, 1 << 24, seed=91)
    ip, ix, w = to_dev(torch, b)
    whole = dmx.dm_sketch(ctx, ip, ix, w, 256, 5)
    assert dmx.dm_sync_status(ctx, raise_on_error=False) == 0
    cuts = [0, 700, 2100, 3000]
    outs, ctxs, streams = [], [], []
    for i in range(3):
        lo, hi = cuts[i], cuts[i + 1]
        sub = b.rows(range(lo, hi))
        c = dmx.dm_create(0)
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            sip, six, sw = to_dev(torch, sub)
            outs.append(dmx.dm_sketch(c, sip, six, sw, 256, 5, stream=s))
        ctxs.append(c)
        streams.append(s)
    for c, s in zip(ctxs, streams):
        assert dmx.dm_sync_status(c, stream=s, raise_on_error=False) == 0
        c.close()
    torch.cuda.synchronize()
    assert torch.equal(torch.cat(outs), whole)


def test_ten_repeats_are_bit_identical(dmx, torch_mod):
    """Concurrent atomicMin in any order gives one minimum: ten runs of each launch form and
    of the LSH and bottom-k sinks repeat their bits exactly."""
    torch = torch_mod
    b = workloads.random_sets(600, 0, 400, 1 << 24, seed=17, scale_lo=1e-3, scale_hi=1e3)
    ip, ix, w = to_dev(torch, b)
    for form in (0, 1, 2):
        c = dmx.dm_create(0)
        dmx.dm_set_option(c, dmx.OPT_FORM, form)
        dmx.dm_set_option(c, dmx.OPT_LARGE_NNZ, 200)
        runs = [dmx.dm_sketch(c, ip, ix, w, 128, 3) for _ in range(10)]
        runs += [dmx.dm_lsh(c, ip, ix, w, 16, 4, 3) for _ in range(10)]
        runs += [dmx.dm_bottomk(c, ip, ix, w, 64, 3) for _ in range(10)]
        assert dmx.dm_sync_status(c, raise_on_error=False) == 0
        for i in (0, 10, 20):
            assert all(torch.equal(runs[i], r) for r in runs[i + 1:i + 10])
        c.close()
