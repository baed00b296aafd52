"""Replica host logic (CPU): shard assignment and the cross-rank reductions
the benchmark uses, run as two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2208_10939_gb300 import sharding


def test_shard_range_covers_every_item_once():
    for n in (0, 1, 7, 4096):
        for w in (1, 2, 3, 8):
            got = [i for r in range(w) for i in sharding.shard_range(n, r, w)]
            assert got == list(range(n))
            sizes = [len(sharding.shard_range(n, r, w)) for r in range(w)]
            assert max(sizes) - min(sizes) <= 1


def test_shard_weighted_balances_uneven_scenes():
    weights = [5000, 200000, 31000, 120000, 8000, 64000, 150000, 20000, 45000, 99000]
    parts = [sharding.shard_weighted(weights, r, 3) for r in range(3)]
    assert sorted(i for p in parts for i in p) == list(range(len(weights)))
    loads = [sum(weights[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(weights)
    assert parts == [sharding.shard_weighted(weights, r, 3) for r in range(3)]   # deterministic


def test_reduce_without_process_group_is_identity():
    assert sharding.reduce_scalar(3.5, "max") == 3.5
    assert sharding.job_throughput(10.0, 2.0)["per_second"] == 5.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = list(sharding.shard_range(10, rank, world))
        work = float(sum(mine))                 # stand-in for echo terms
        secs = 1.0 + rank                       # rank 1 is slower
        res = sharding.job_throughput(work, secs)
        q.put((rank, mine, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_work_and_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    assert out[0][1] == [0, 1, 2, 3, 4] and out[1][1] == [5, 6, 7, 8, 9]
    for _, _, res in out:
        assert res["work"] == 45.0 and res["seconds"] == 2.0
        assert res["per_second"] == 22.5
