"""The multi-rank path on CPU: world size 2 over gloo (127.0.0.1)."""
import os

import pytest
import torch.multiprocessing as mp

from paper_2411_08962_gb300 import sharding


def test_shard_partitions_items():
    for n in (0, 1, 7, 64):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                seen += list(sharding.shard(n, r, world))
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        sharding.shard(4, 2, 2)


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = list(sharding.shard(64, rank, world))
    seeds = [sharding.config_seed(100, i) for i in mine]
    slowest = sharding.max_over_ranks(10.0 + rank)            # per-rank "elapsed ms"
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    if rank == 0:
        out.put((slowest, gathered))
    dist.destroy_process_group()


def test_two_ranks_over_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    slowest, gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == 11.0
    flat = gathered[0] + gathered[1]
    assert flat == [sharding.config_seed(100, i) for i in range(64)] and len(set(flat)) == 64
