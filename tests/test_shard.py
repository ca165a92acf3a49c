"""Multi-process host logic on the CPU: two gloo ranks partition the work
without overlap and reduce time (max) and work (sum) as the benchmark does."""
import os
import socket

import pytest

from paper_1508_02892_gb300 import shard


def test_rank_share_partitions_the_requests():
    items = list(range(23))
    parts = [shard.rank_share(items, r, 3) for r in range(3)]
    assert sorted(sum(parts, [])) == items
    assert all(not set(a) & set(b) for i, a in enumerate(parts) for b in parts[i + 1:])
    with pytest.raises(ValueError):
        shard.rank_share(items, 3, 3)


def test_instance_seeds_differ_by_rank():
    assert len({shard.instance_seed(r) for r in range(8)}) == 8
    assert shard.instance_seed(0) == 2026


def test_aggregate_without_process_group_is_local():
    assert shard.aggregate(3.5, 10) == (3.5, 10.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = list(range(10))
        mine = shard.rank_share(items, rank, world)
        ms_local = 100.0 + 7.0 * rank       # rank 1 is the slowest
        n_local = float(sum(mine))          # its share of the work
        out[rank] = shard.aggregate(ms_local, n_local)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r] == (107.0, float(sum(range(10))))
