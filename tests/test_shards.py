"""Shot sharding over ranks (the multi-process path has no data collective): every shot is
owned by exactly one rank, blocks are balanced, and the timing reduction takes the max.
Two gloo ranks on the CPU."""

import os

import pytest

from paper_1304_3542_gb300.shards import shard_shots


@pytest.mark.parametrize("nshots,world", [(64, 1), (64, 2), (64, 3), (7, 4), (3, 8), (0, 2)])
def test_every_shot_owned_once_and_balanced(nshots, world):
    owned = [shard_shots(nshots, r, world) for r in range(world)]
    flat = [s for o in owned for s in o]
    assert sorted(flat) == list(range(nshots))
    sizes = [len(o) for o in owned]
    assert max(sizes) - min(sizes) <= 1
    for o in owned:
        assert o == list(range(o[0], o[0] + len(o))) if o else True


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1304_3542_gb300.shards import max_over_ranks, shard_shots

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_shots(10, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = max_over_ranks(1.5 + rank)
    q.put((rank, gathered, t))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in res:
        assert sorted(s for g in gathered for s in g) == list(range(10))
        assert t == 2.5
