"""GPU parity of dm_compare (similarity counts of sketches, Section 1.1) with the oracle's
slot-by-slot counts: exact integers for keys and every b, row-aligned pairs and the cross form,
k not a multiple of the warp or tile sizes, and sketches made by the library itself."""
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


@pytest.fixture(scope="module")
def ctx(dmx):
    c = dmx.dm_create(0)
    yield c
    c.close()


def dev(torch, arr):
    return torch.from_numpy(np.ascontiguousarray(arr).view(np.int64)).cuda()


def random_sketches(rng, n, k, bits, agree):
    """Pairs of rows agreeing on a fraction `agree` of their slots."""
    if bits == 0:
        a = rng.integers(0, 2 ** 63, size=(n, k), dtype=np.uint64)
        c = a.copy()
        flip = rng.random((n, k)) > agree
        c[flip] ^= np.uint64(1) << np.uint64(40)
        return a, c
    W = (k * bits + 63) // 64
    a = rng.integers(0, 2 ** 63, size=(n, W), dtype=np.uint64) | (rng.integers(0, 2, size=(n, W), dtype=np.uint64) << np.uint64(63))
    c = a ^ (rng.random((n, W)) > agree).astype(np.uint64) * rng.integers(0, 2 ** 63, size=(n, W), dtype=np.uint64)
    used = k * bits - 64 * (W - 1)
    if used < 64:
        a[:, -1] &= np.uint64((1 << used) - 1)
        c[:, -1] &= np.uint64((1 << used) - 1)
    return a, c


@pytest.mark.parametrize("bits", [0, 1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("k", [1, 37, 64, 256, 1000])
def test_pairs_and_cross_parity(dmx, torch_mod, ctx, oracle_mod, bits, k):
    rng = np.random.default_rng(1000 * bits + k)
    a, c = random_sketches(rng, 300, k, bits, 0.6)
    got = dmx.dm_compare(ctx, dev(torch_mod, a), dev(torch_mod, c), k, bits=bits)
    exp = oracle_mod.compare(a, c, k, bits=bits)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)
    kc = k if bits == 0 else min(k, 64 * 64 // bits)    # the cross form takes b-bit rows of <= 64 words
    a, c = random_sketches(rng, 70, kc, bits, 0.6)
    na, nc = 45, 70                                     # ragged tiles on both sides
    got = dmx.dm_compare(ctx, dev(torch_mod, a[:na]), dev(torch_mod, c[:nc]), kc, bits=bits, cross=True)
    exp = oracle_mod.compare(a[:na], c[:nc], kc, bits=bits, mode="cross")
    assert np.array_equal(got.cpu().numpy().view(np.uint32), exp)


def test_library_sketches_estimate_jaccard(dmx, torch_mod, ctx, oracle_mod):
    """dm_sketch / dm_sketch_bbit of pair batches, compared on the GPU: the counts equal the
    oracle's on the oracle's sketches, and the estimates center on the exact J."""
    torch = torch_mod
    rng = np.random.default_rng(8)
    pairs = [workloads.similar_pair(rng, 32, 2 * 0.5 / 1.5) for _ in range(2000)]
    xs = workloads.csr_of([(p[0], p[1]) for p in pairs])
    ys = workloads.csr_of([(p[2], p[3]) for p in pairs])

    def to_dev(b):
        return (torch.from_numpy(b.indptr).cuda(), torch.from_numpy(b.indices.view(np.int32)).cuda(),
                torch.from_numpy(b.weights).cuda())

    k = 128
    sx = dmx.dm_sketch(ctx, *to_dev(xs), k, 3)
    sy = dmx.dm_sketch(ctx, *to_dev(ys), k, 3)
    m = dmx.dm_compare(ctx, sx, sy, k).cpu().numpy().view(np.uint32)
    ox = oracle_mod.sketch(xs.indptr, xs.indices, xs.weights, k, 3, threads=16)
    oy = oracle_mod.sketch(ys.indptr, ys.indices, ys.weights, k, 3, threads=16)
    assert np.array_equal(m, oracle_mod.compare(ox, oy, k))
    est = dmx.estimate_jaccard(dmx.dm_compare(ctx, sx, sy, k), k).cpu().numpy()
    assert np.array_equal(est, oracle_mod.estimate_jaccard(m, k))          # the same binary64 steps
    assert abs(est.mean() - 0.5) < 0.01
    wx = dmx.dm_sketch_bbit(ctx, *to_dev(xs), k, 1, 3)
    wy = dmx.dm_sketch_bbit(ctx, *to_dev(ys), k, 1, 3)
    m1 = dmx.dm_compare(ctx, wx, wy, k, bits=1).cpu().numpy().view(np.uint32)
    est1 = dmx.estimate_jaccard(dmx.dm_compare(ctx, wx, wy, k, bits=1), k, bits=1).cpu().numpy()
    assert np.array_equal(est1, oracle_mod.estimate_jaccard(m1, k, bits=1))
    assert abs(est1.mean() - 0.5) < 0.02
    for b in (2, 4, 8, 16, 32):                         # every b-bit correction, on all counts 0..k
        mm = np.arange(k + 1, dtype=np.uint32)
        got = dmx.estimate_jaccard(torch.from_numpy(mm.view(np.int32)).cuda(), k, bits=b).cpu().numpy()
        assert np.array_equal(got, oracle_mod.estimate_jaccard(mm, k, bits=b))
    cross = dmx.dm_compare(ctx, sx[:50], sy[:60], k, cross=True).cpu().numpy().view(np.uint32)
    assert np.array_equal(np.diag(cross[:50, :50]), m[:50])


def test_compare_rejects_bad_arguments(dmx, torch_mod, ctx):
    a = torch_mod.zeros((4, 8), dtype=torch_mod.int64, device="cuda")
    c = torch_mod.zeros((5, 8), dtype=torch_mod.int64, device="cuda")
    with pytest.raises(ValueError):
        dmx.dm_compare(ctx, a, c, 8)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_compare(ctx, a, a, 8, bits=3)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_compare(ctx, a, a, 0)


@pytest.mark.parametrize("bits", [0, 1, 8])
@pytest.mark.parametrize("nc", [5, 70, 3000])
def test_topk_parity(dmx, torch_mod, ctx, oracle_mod, bits, nc):
    """dm_compare_topk against the oracle's stable selection: counts drawn from a small alphabet,
    so many candidates tie and the row order decides; n_c below topk, within one tile, and over
    several spans of c (folded by the merge kernel); query rows ragged against the tile."""
    rng = np.random.default_rng(77 + bits + nc)
    k, na = (37 if bits == 0 else 64), 45
    if bits == 0:
        a = rng.integers(0, 3, size=(na, k), dtype=np.uint64)
        c = rng.integers(0, 3, size=(nc, k), dtype=np.uint64)
    else:
        W = (k * bits + 63) // 64
        pat = rng.integers(0, 2 ** 63, size=(4, W), dtype=np.uint64)     # few distinct words: ties
        a = pat[rng.integers(0, 4, size=(na, W)), np.arange(W)]
        c = pat[rng.integers(0, 4, size=(nc, W)), np.arange(W)]
    for topk in (1, 7, 32):
        rows, counts = dmx.dm_compare_topk(ctx, dev(torch_mod, a), dev(torch_mod, c), k, topk, bits=bits)
        er, ec = oracle_mod.compare_topk(a, c, k, topk, bits=bits)
        assert np.array_equal(rows.cpu().numpy().view(np.uint32), er), (bits, nc, topk)
        assert np.array_equal(counts.cpu().numpy().view(np.uint32), ec), (bits, nc, topk)


def test_topk_many_spans_and_library_sketches(dmx, torch_mod, ctx, oracle_mod):
    """Sketches made by dm_sketch: 5 queries against 50,000 candidates (many spans) that include
    a copy of each query and a J = 0.9 neighbour; the result equals the oracle's selection and
    ranks the copy first with all k slots agreeing."""
    torch = torch_mod
    rng = np.random.default_rng(31)
    k = 64
    base = workloads.random_sets(50_000 - 10, 10, 60, 1 << 20, seed=41)
    q_rows, near_rows = [], []
    for _ in range(5):
        ix, wx, iy, wy = workloads.similar_pair(rng, 40, 2 * 0.9 / 1.9)
        q_rows.append((ix, wx))
        near_rows.append((iy, wy))
    qb = workloads.csr_of(q_rows)
    rows_c = [(base.indices[base.indptr[i]:base.indptr[i + 1]], base.weights[base.indptr[i]:base.indptr[i + 1]])
              for i in range(base.n_sets)] + near_rows + q_rows
    cb = workloads.csr_of(rows_c)

    def sketch(b):
        return dmx.dm_sketch(ctx, torch.from_numpy(b.indptr).cuda(), torch.from_numpy(b.indices.view(np.int32)).cuda(),
                             torch.from_numpy(b.weights).cuda(), k, 4)

    qa, ca = sketch(qb), sketch(cb)
    rows, counts = dmx.dm_compare_topk(ctx, qa, ca, k, 10)
    er, ec = oracle_mod.compare_topk(qa.cpu().numpy().view(np.uint64), ca.cpu().numpy().view(np.uint64), k, 10)
    assert np.array_equal(rows.cpu().numpy().view(np.uint32), er)
    assert np.array_equal(counts.cpu().numpy().view(np.uint32), ec)
    n0 = base.n_sets
    for i in range(5):
        assert ec[i, 0] == k and n0 + 5 + i in er[i, :2]           # the copy (the neighbour may tie it)
        assert n0 + i in er[i, :3]


def test_topk_rejects_bad_arguments(dmx, torch_mod, ctx):
    a = torch_mod.zeros((4, 16), dtype=torch_mod.int64, device="cuda")
    for topk in (0, 33):
        with pytest.raises(dmx.DartMinHashError):
            dmx.dm_compare_topk(ctx, a, a, 16, topk)
    with pytest.raises(dmx.DartMinHashError):
        dmx.dm_compare_topk(ctx, a, a, 16, 4, bits=3)
    rows, counts = dmx.dm_compare_topk(ctx, a, a[:0], 16, 4)             # no candidates
    assert np.all(rows.cpu().numpy().view(np.uint32) == 0xFFFFFFFF) and not counts.any()
