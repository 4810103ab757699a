"""Multi-GPU use: fields are independent and field b of a call is keyed by
seed + b, so ranks split a job into contiguous field ranges and need no
collective on the data path.  Only timing uses one (the maximum over ranks).
No GPU code here; the helpers run with any torch.distributed backend."""
from __future__ import annotations


def field_range(rank: int, world: int, total: int):
    """Contiguous share [start, stop) of `total` fields for `rank` of `world`;
    the first total % world ranks take one extra field."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int, world: int, total: int) -> int:
    """Seed whose fields 0.. are the global fields of this rank's range:
    global field b has key seed + b, so the range [start, stop) starts at seed + start."""
    return seed + field_range(rank, world, total)[0]


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank number (e.g. elapsed time) over all ranks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
