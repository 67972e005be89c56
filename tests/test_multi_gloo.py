"""Multi-process host logic of the replica path on CPU (gloo, world size 2)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_11520_b300.shard import column_shard, rank_seed, request_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_2609_11520_b300.shard import column_shard, max_over_ranks, request_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, cnt = column_shard(67, world, rank)
    t = max_over_ranks(1.5 + rank, dist)
    reqs = request_shard(list(range(11)), world, rank)
    dist.barrier()
    q.put((rank, start, cnt, t, reqs))
    dist.destroy_process_group()


def test_column_shard_covers_exactly():
    for k in (0, 1, 63, 64, 67):
        for world in (1, 2, 3, 8):
            got = [column_shard(k, world, r) for r in range(world)]
            assert sum(c for _, c in got) == k
            pos = 0
            for s, c in got:
                assert s == pos
                pos += c
    with pytest.raises(ValueError):
        column_shard(4, 2, 2)


def test_request_shard_and_seeds():
    ids = list(range(10))
    parts = [request_shard(ids, 3, r) for r in range(3)]
    assert sorted(sum(parts, [])) == ids
    assert len({rank_seed(7, r) for r in range(8)}) == 8


def test_two_ranks_gloo():
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
    assert [(s, c) for _, s, c, _, _ in res] == [(0, 34), (34, 33)]
    assert all(t == 2.5 for _, _, _, t, _ in res)             # max over ranks
    assert sorted(res[0][4] + res[1][4]) == list(range(11))
