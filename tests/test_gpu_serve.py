"""GPU tests of the serving loop (dm_server_*): every request, whatever batch, lane or form it
runs in, gets exactly the keys of its row computed alone (checked against the oracle), and the
failure paths (bad input, out-of-range rows, an injected batch failure, over-budget and
oversized requests) answer per request while the server carries on."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

THREADS = 16


@pytest.fixture(scope="module")
def dmx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2005_11547_gb300 as dmx
    dmx.build()
    dmx.load()
    return dmx


def trace(n, seed, max_nnz=100_000):
    """W4-like requests (the serving workload's sizes): nnz = min(max_nnz, floor(Pareto(1.2) + 1)),
    weights U(0, 5], k uniform over {64, 256, 1024}, seeds 1 or 2, arrivals at 50,000/s.  The
    first request and one in the middle have the largest nnz the workload allows (100,000) with
    k = 1024, so they run alone at the start and in the mix later."""
    rng = np.random.default_rng(seed)
    lens = np.minimum(max_nnz, np.floor(rng.pareto(1.2, size=n) + 1.0)).astype(np.int64)
    lens[:3] = [100_000, 3000, 2100]           # sets for the block-per-set path
    lens[n // 2] = 100_000
    ip = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=ip[1:])
    idx = workloads._ragged_distinct(rng, lens, 1 << 24)
    w = (5.0 * (1.0 - rng.random(int(ip[-1])))).astype(np.float32)
    ks = rng.choice(np.array([64, 256, 1024], dtype=np.int32), size=n)
    ks[0] = ks[n // 2] = 1024
    seeds = rng.integers(1, 3, size=n).astype(np.uint64)
    arr = np.cumsum(rng.exponential(1.0 / 50_000, size=n) * 1e9).astype(np.int64)
    return ip, idx, w, ks, seeds, arr


def oracle_per_request(oracle_mod, ip, idx, w, ks, seeds):
    """Keys of every request, computed by the oracle one (k, seed) group at a time."""
    res = [None] * (len(ip) - 1)
    for k in np.unique(ks):
        for s in np.unique(seeds):
            sel = np.nonzero((ks == k) & (seeds == s))[0]
            if len(sel) == 0:
                continue
            rows = [(idx[ip[i]:ip[i + 1]], w[ip[i]:ip[i + 1]]) for i in sel]
            b = workloads.csr_of(rows)
            out = oracle_mod.sketch(b.indptr, b.indices, b.weights, int(k), int(s), threads=THREADS)
            for j, i in enumerate(sel):
                res[i] = out[j]
    return res


@pytest.mark.parametrize("mode", ["batched", "window", "per_request"])
def test_replay_matches_oracle(dmx, oracle_mod, mode):
    ip, idx, w, ks, seeds, arr = trace(1500, 4)
    kw = {"batched": dict(lanes=4), "window": dict(lanes=2, max_wait_us=300),
          "per_request": dict(lanes=1, per_request=True)}[mode]
    srv = dmx.Server(0, **kw)
    out, lat, st = srv.replay(ip, idx, w, ks, seeds, arr)
    stats = srv.stats()
    srv.close()
    assert np.all(st == 0)
    assert np.all(lat > 0)
    assert stats["completed"] == 1500 and stats["failed"] == 0
    if mode == "per_request":
        assert stats["mean_batch"] == 1.0
    exp = oracle_per_request(oracle_mod, ip, idx, w, ks, seeds)
    off = np.concatenate([[0], np.cumsum(ks.astype(np.int64))])
    for i in range(1500):
        got = out[off[i]:off[i + 1]]
        assert np.array_equal(got, exp[i]), f"request {i} (k={ks[i]}, nnz={ip[i + 1] - ip[i]})"


def test_tickets_from_threads_match_dm_sketch(dmx, oracle_mod):
    """Submissions from several host threads; each result equals the oracle's for its row."""
    import threading
    ip, idx, w, ks, seeds, _ = trace(600, 5)
    srv = dmx.Server(0, lanes=3)
    outs = [None] * 600
    errors = []

    def client(t):
        try:
            tickets = []
            for i in range(t, 600, 4):
                while True:
                    rc, tk, o = srv.submit(idx[ip[i]:ip[i + 1]].copy(), w[ip[i]:ip[i + 1]].copy(), int(ks[i]),
                                           int(seeds[i]))
                    if rc == 0:
                        break
                tickets.append((i, tk, o))
            for i, tk, o in tickets:
                assert srv.wait(tk) == 0
                outs[i] = o
        except Exception as e:     # surfaced below
            errors.append(e)

    th = [threading.Thread(target=client, args=(t,)) for t in range(4)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    srv.close()
    assert not errors, errors
    exp = oracle_per_request(oracle_mod, ip, idx, w, ks, seeds)
    for i in range(600):
        assert np.array_equal(outs[i], exp[i]), f"request {i}"


def test_failures_are_per_request(dmx, oracle_mod):
    srv = dmx.Server(0, lanes=1, max_wait_us=2000)
    good = (np.array([5, 9, 11], np.uint32), np.array([0.5, 1.0, 2.0], np.float32))
    # host checks: NaN / negative weight, bad k
    for bad in (np.array([0.5, np.nan, 1.0], np.float32), np.array([0.5, -1.0, 1.0], np.float32)):
        with pytest.raises(dmx.DartMinHashError) as e:
            srv.submit(good[0], bad, 64, 1)
        assert e.value.code == 1
    with pytest.raises(dmx.DartMinHashError):
        srv.submit(good[0], good[1], 0, 1)
    # a row out of the supported range (t x_i >= 2^39 - 1) fails alone; its batch-mates succeed
    _, t1, o1 = srv.submit(good[0], good[1], 64, 1)
    _, t2, o2 = srv.submit(good[0], np.array([0.5, 1e30, 2.0], np.float32), 64, 1)
    _, t3, o3 = srv.submit(np.zeros(0, np.uint32), np.zeros(0, np.float32), 64, 1)   # empty set: sentinel
    assert srv.wait(t1) == 0 and srv.wait(t2) == 5 and srv.wait(t3) == 0
    assert np.all(o3 == np.uint64(2 ** 64 - 1))
    b = workloads.csr_of([good])
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, 64, 1)[0]
    assert np.array_equal(o1, exp)
    # injected launch failure: the next batch fails, later ones succeed
    srv.fail_batches(1)
    _, t4, _ = srv.submit(good[0], good[1], 64, 1)
    assert srv.wait(t4) == 3
    _, t5, o5 = srv.submit(good[0], good[1], 64, 1)
    assert srv.wait(t5) == 0 and np.array_equal(o5, exp)
    # a request larger than a lane is refused outright
    small = dmx.Server(0, lanes=1, mem_budget_bytes=1 << 20)
    n = (1 << 20) // 8
    with pytest.raises(dmx.DartMinHashError) as e:
        small.submit(np.arange(n, dtype=np.uint32), np.ones(n, np.float32), 64, 1)
    assert e.value.code == 2
    small.close()
    st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 5
    srv.close()


def test_admission_budget_holds(dmx, oracle_mod):
    """A 1 MiB budget with requests of 160 KB: submissions beyond the budget are refused with
    EAGAIN and succeed on retry; every result is still exact."""
    rng = np.random.default_rng(8)
    srv = dmx.Server(0, lanes=1, mem_budget_bytes=1 << 20)
    rows, outs, tickets = [], [], []
    eagain = 0
    for i in range(40):
        idx = np.sort(rng.choice(1 << 24, 20000, replace=False)).astype(np.uint32)
        wt = (5.0 * (1.0 - rng.random(20000))).astype(np.float32)
        rows.append((idx, wt))
        while True:
            rc, tk, o = srv.submit(idx, wt, 256, 3)
            if rc == 0:
                break
            eagain += 1
        tickets.append(tk)
        outs.append(o)
    for tk in tickets:
        assert srv.wait(tk) == 0
    st = srv.stats()
    srv.close()
    assert st["rejected"] == eagain
    b = workloads.csr_of(rows)
    exp = oracle_mod.sketch(b.indptr, b.indices, b.weights, 256, 3, threads=THREADS)
    for i in range(40):
        assert np.array_equal(outs[i], exp[i])
