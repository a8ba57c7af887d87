"""Multi-rank placement of independent boxes, checked with world_size-2
gloo process groups on the CPU (no GPU): every box on exactly one rank,
balanced loads, and the max-over-ranks timing reduction."""
import os

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2105_01865_gb300.sharding import lpt_assign, max_over_ranks


def test_lpt_partition_and_balance():
    costs = [n ** 3 for n in (32, 48, 64, 96, 128, 128, 96, 32, 64, 48, 128, 96, 32)]
    for world in (1, 2, 3, 4, 8):
        parts = lpt_assign(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(costs)
    with pytest.raises(ValueError):
        lpt_assign(costs, 0)


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = lpt_assign(costs, world)
        mine = parts[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(0.5 + rank)
        out[rank] = (gathered, t)
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    costs = [32 ** 3, 128 ** 3, 64 ** 3, 96 ** 3, 48 ** 3, 128 ** 3, 32 ** 3]
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, costs, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        gathered, t = res[rank]
        assert sorted(i for p in gathered for i in p) == list(range(len(costs)))
        assert gathered == lpt_assign(costs, world)
        assert t == 1.5
