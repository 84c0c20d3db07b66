"""Multi-rank host logic on CPU with the gloo backend (world size 2): shard
ranges, per-rank seeds and the max-over-ranks timing reduction used by
bench.py under torchrun.  The data path itself has no collective."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2602_24271_b300.sharding import ct_shard, max_over_ranks, rank_seed


def test_ct_shard_partitions_exactly():
    for n in (0, 1, 7, 2048, 8193):
        for w in (1, 2, 3, 8):
            ranges = [ct_shard(n, w, r) for r in range(w)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and b >= a
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        ct_shard(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, end = ct_shard(2048 * world, world, rank)
    local_ms = 100.0 + 17.0 * rank  # rank 1 is the slow one
    ms = max_over_ranks(local_ms, dist)
    q.put((rank, start, end, rank_seed(1, rank), ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [(r[1], r[2]) for r in res] == [(0, 2048), (2048, 4096)]
    assert res[0][3] != res[1][3]
    assert all(r[4] == 117.0 for r in res)  # both ranks report the slowest rank's time
