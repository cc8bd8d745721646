"""Shot-parallel work split for several processes (one GPU each).

Shots are independent problems (each has its own initial data and eps and shares only
the velocity), so N ranks take disjoint, contiguous, balanced blocks of the shot list
and need no collective on the data path; only the timing is reduced (max over ranks).
"""

from __future__ import annotations

from typing import List


def shard_shots(nshots: int, rank: int, world: int) -> List[int]:
    """Shot indices of rank `rank` out of `world`: contiguous blocks whose sizes differ by
    at most one, in rank order."""
    if world < 1 or not (0 <= rank < world) or nshots < 0:
        raise ValueError("need 0 <= rank < world and nshots >= 0")
    base, extra = divmod(nshots, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (value itself when no
    group is initialised)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
