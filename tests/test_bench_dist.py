"""The bench's N > 1 host logic on CPU: two gloo ranks (one process each),
the whole-job aggregation (sum of work, max of time over ranks) and the
per-rank problems (independent seeds: weak scaling, no data collective)."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        agg = bench.aggregate(dist, 10 * (rank + 1), 100.0 + rank, "cpu")
        _, x_true, z = bench.make_problem(synth.get_config("c8"), rank)
        q.put((rank, agg, float(x_true.sum()), float(z[:8].sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_and_draw_independent_problems():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, agg, xs, zs = q.get(timeout=120)
        out[rank] = (agg, xs, zs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the whole-job figures: 10 + 20 evaluations over max(100, 101) ms
    assert out[0][0] == out[1][0] == (30.0, 101.0)
    # each rank solves its own seeded problem (phantom and noise differ)
    assert out[0][1] != out[1][1] and out[0][2] != out[1][2]


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.aggregate(None, 7, 12.5, "cpu") == (7.0, 12.5)
