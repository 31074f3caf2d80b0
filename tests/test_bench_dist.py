"""bench.py's multi-rank host logic (barrier, max and sum over ranks) on a world-size-2
gloo group on the CPU: the timing reduction is the max over ranks and the unit count is
the sum."""
import os
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, _ = bench.dist_env()
    dist = bench.dist_init(w, use_cuda=False)
    bench.barrier(dist, use_cuda=False)
    t = bench.max_over_ranks(dist, 1.0 + r, use_cuda=False)
    n = bench.sum_over_ranks(dist, 1000.0 * (r + 1), use_cuda=False)
    q.put((r, t, n))
    dist.destroy_process_group()


def test_two_rank_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2.0, 3000.0), (1, 2.0, 3000.0)]
