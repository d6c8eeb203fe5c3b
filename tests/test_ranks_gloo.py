"""The multi-rank host path on CPU: two gloo ranks split the 96-domain ensemble with
shard_domains and reduce a step time with max_over_ranks; the shards must partition the
domains (each exactly once), balance their cells, and agree on every rank."""
import os
import socket

import pytest

from paper_1901_02955_gb300.ranks import max_over_ranks, shard_domains

SIZES = [n * n for n in (64, 128, 256, 512) for _ in range(24)]


def test_shards_partition_and_balance():
    for world in (1, 2, 3, 4, 8):
        shards = shard_domains(SIZES, world)
        flat = sorted(d for s in shards for d in s)
        assert flat == list(range(len(SIZES)))
        loads = [sum(SIZES[d] for d in s) for s in shards]
        assert max(loads) <= 1.05 * sum(SIZES) / world + max(SIZES)
    assert shard_domains(SIZES, 1) == [list(range(len(SIZES)))]
    with pytest.raises(ValueError):
        shard_domains(SIZES, 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard_domains(SIZES, world)[rank]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(1.0 + rank, dist)
        q.put((rank, mine, gathered, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_ensemble():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == list(range(len(SIZES)))
    for _, _, gathered, t in res:
        assert gathered == shards  # every rank sees the same partition
        assert t == 2.0  # the slowest rank's time
    assert max_over_ranks(3.5) == 3.5  # no process group: the value itself
