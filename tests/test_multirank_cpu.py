"""The multi-rank logic of bench.py on CPU with two gloo ranks: every rank
owns a distinct dataset, batch shards partition the datasets, and the job
time is the maximum over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        seeds = [None] * world
        dist.all_gather_object(seeds, bench.dataset_seed(rank))
        shards = [None] * world
        dist.all_gather_object(shards, bench.shard(11, world, rank))
        out[rank] = (t, seeds, shards)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, seeds, shards = res[r]
        assert t == 15.0                                  # max over ranks
        assert len(set(seeds)) == world                   # independent datasets
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(11))                    # shards partition the batch
        assert abs(len(shards[0]) - len(shards[1])) <= 1


@pytest.mark.parametrize("count,world", [(0, 3), (5, 8), (256, 8), (64, 3)])
def test_shards_partition(count, world):
    parts = [bench.shard(count, world, r) for r in range(world)]
    assert sorted(i for s in parts for i in s) == list(range(count))
