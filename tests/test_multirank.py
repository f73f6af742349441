"""Host logic of the multi-rank benchmark on CPU: two gloo ranks (one process each) combine their
timings by max and their work by sum, draw disjoint scene seeds, and split one scene into point
ranges that tile it (no GPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.reduce_over_ranks(10.0 + 5.0 * rank, dist, "cpu")            # per-rank step time
        pts = bench.reduce_over_ranks(1000 * (rank + 1), dist, "cpu", "sum")   # per-rank points
        # one scene split over the ranks: the gathered ranges tile [0, n) exactly, in rank order
        import torch
        n = 1000003
        lo, hi = bench.rank_range(n, rank, world)
        got = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(got, torch.tensor([lo, hi], dtype=torch.int64))
        bounds = [tuple(int(v) for v in t) for t in got]
        out.put((rank, ms, pts, bench.rank_first_seed(rank), bench.dist_env(), bounds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_seed():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, pts, seed, env, bounds in res:
        assert ms == 15.0             # the slowest rank's time
        assert pts == 3000.0          # all ranks' points
        assert env == (rank, world, 0)
        assert bounds[0][0] == 0 and bounds[-1][1] == 1000003
        assert all(bounds[q][1] == bounds[q + 1][0] for q in range(world - 1))
        assert max(h - l for l, h in bounds) - min(h - l for l, h in bounds) <= 1
    seeds = [r[3] for r in res]
    # the serving batches of different ranks (16 consecutive seeds each) do not overlap
    assert len(set(seeds)) == world and abs(seeds[1] - seeds[0]) >= 16


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.rank_first_seed(0) == 200
