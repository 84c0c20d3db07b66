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


def _agg_worker(rank, world, port, q):
    """Each rank reduces its shard of a 4-ciphertext column to one partial
    aggregate (oracle, N = 16), the partials are all-gathered over gloo and
    added mod Q; the total must decrypt to the sum of the whole column."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    from paper_2602_24271_b300.sharding import allgather_partials

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    o = oracle.Oracle(4)
    o.keygen(7)
    for g in o.galois_elements():
        o.galois_keygen(5, g)
    x = np.random.default_rng(40).integers(0, 65537, 4 * o.N).astype(np.uint32)  # same column on every rank
    start, end = ct_shard(4, world, rank)
    mine = np.stack([o.encrypt(x[c * o.N:(c + 1) * o.N], 41, c) for c in range(start, end)])
    part = o.rotate_sum(o.linear(mine, [1] * len(mine)))
    gathered = allgather_partials(torch.from_numpy(part.view(np.int64)), dist).numpy().view(np.uint64)
    total = o.linear(gathered, [1] * world)
    q.put((rank, gathered.shape[0], int(o.decrypt(total)[0]), int(x.astype(np.int64).sum() % 65537),
           bool(np.all(o.decrypt(total) == o.decrypt(total)[0]))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_partial_aggregates():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_agg_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, n, got, want, uniform in res:
        assert n == world and got == want and uniform
