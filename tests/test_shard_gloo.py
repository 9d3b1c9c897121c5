"""Multi-rank host logic on CPU: two gloo ranks split the 256-grain batch, check that the
shards cover every system exactly once and are balanced, and combine timings with the
max-over-ranks reduction the benchmark uses."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1310_6143_gb300.shard import rank_systems, shard_systems


def _worker(rank, world, port, sizes, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = rank_systems(sizes, rank, world)
    spins = torch.tensor([sum(sizes[k] for k in mine)], dtype=torch.int64)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)  # per-rank time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total = spins.clone()
    dist.all_reduce(total, op=dist.ReduceOp.SUM)
    if rank == 0:
        q.put((gathered, float(t.item()), int(total.item())))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_batch():
    import numpy as np

    sizes = [int(v) for v in np.random.default_rng(12345).integers(2000, 40001, 256)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(k for part in gathered for k in part)
    assert flat == list(range(256))
    loads = [sum(sizes[k] for k in part) for part in gathered]
    assert abs(loads[0] - loads[1]) <= max(sizes)
    assert tmax == 2.0 and total == sum(sizes)


def test_shard_single_rank_and_many():
    sizes = [5, 1, 9, 3]
    assert shard_systems(sizes, 1) == [[0, 1, 2, 3]]
    parts = shard_systems(sizes, 3)
    assert sorted(k for p in parts for k in p) == [0, 1, 2, 3]
    with pytest.raises(ValueError):
        shard_systems(sizes, 0)
