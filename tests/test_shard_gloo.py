"""Multi-rank host logic on CPU (gloo, world size 2): the field ranges cover a
job exactly once, rank seeds reproduce the global keys, and the timing
reduction takes the maximum over ranks."""
import os
import socket

import pytest

from paper_1105_2737_gb300.shard import field_range, rank_seed


@pytest.mark.parametrize("world,total", [(1, 64), (2, 64), (3, 64), (4, 7), (8, 4096), (5, 3)])
def test_field_ranges_partition(world, total):
    seen = []
    for r in range(world):
        a, b = field_range(r, world, total)
        assert 0 <= a <= b <= total
        seen.extend(range(a, b))
    assert seen == list(range(total))


def test_rank_seed_matches_global_keys():
    seed, world, total = 1000, 3, 10
    keys = []
    for r in range(world):
        a, b = field_range(r, world, total)
        s = rank_seed(seed, r, world, total)
        keys.extend(s + i for i in range(b - a))
    assert keys == [seed + b for b in range(total)]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    from paper_1105_2737_gb300.shard import max_over_ranks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, max_over_ranks(10.0 + rank), field_range(rank, world, 64)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert all(p.exitcode == 0 for p in ps)
    assert [r[1] for r in res] == [11.0, 11.0]
    assert [r[2] for r in res] == [(0, 32), (32, 64)]
