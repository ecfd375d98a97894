"""Multi-rank host logic: column shards and the max-over-ranks timing reduction, run as
world_size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2004_13904_gb300.parallel import max_over_ranks, shard_columns


@pytest.mark.parametrize("total,world", [(1260, 1), (1260, 2), (2510, 4), (7, 3), (0, 2), (2, 5)])
def test_shards_partition_columns(total, world):
    shards = [shard_columns(total, world, r) for r in range(world)]
    assert sum(c for _, c in shards) == total
    pos = 0
    for first, count in shards:
        assert first == pos and count >= 0
        pos += count
    counts = [c for _, c in shards]
    assert max(counts) - min(counts) <= 1


def test_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shard_columns(10, 0, 0)
    with pytest.raises(ValueError):
        shard_columns(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = shard_columns(1261, world, rank)
        elapsed = 10.0 + rank * 3.5          # each rank's own timing
        out[rank] = (first, count, max_over_ranks(elapsed))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_reduction():
    ctx = mp.get_context("spawn")
    world = 2
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world,
                           start_method="spawn", join=True)
        res = dict(out)
    assert res[0][:2] == (0, 631) and res[1][:2] == (631, 630)
    assert res[0][2] == res[1][2] == 13.5      # every rank sees the slowest rank's time


def test_max_over_ranks_single_process():
    assert max_over_ranks(4.25) == 4.25
