"""Multi-rank member sharding on CPU ranks (gloo, world size 2): the split
covers every member once, results gather in member order, and the timing
reduction takes the slowest rank -- the host-side logic of `bench.py --gpus N`
and of sharded batches."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1907_00908_gb300 import shard


def test_assign_covers_every_member_once():
    costs = [512 ** 3] + [128 ** 3] * 64 + [n ** 3 for n in range(48, 161, 7)]
    for world in (1, 2, 3, 8):
        parts = shard.assign(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / world + max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.assign(costs, world)[rank]
    # stand-in for the per-member run: a deterministic function of the index
    vals = [[i, 2.0 * i, float(i) ** 0.5] for i in mine]
    res = shard.gather_results(mine, vals, len(costs), dist)
    t = shard.max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        q.put((res.tolist(), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_gather_and_time():
    costs = [5, 1, 4, 1, 5, 9, 2, 6, 5]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = [[i, 2.0 * i, float(i) ** 0.5] for i in range(len(costs))]
    np.testing.assert_allclose(res, expect)
    assert t == 2.0
