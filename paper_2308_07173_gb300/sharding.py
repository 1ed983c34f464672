"""Host-side sharding of scans over ranks (one GPU per rank).

Queries are independent, so whole scans are dealt out round-robin and each
rank answers its own against its own copy of the map; no data crosses
ranks.  Only timing is reduced (max over ranks) and counts summed, through
torch.distributed when it is initialised (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import List


def scans_for_rank(n_scans: int, world: int, rank: int) -> List[int]:
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    return list(range(rank, n_scans, world))


def _reduce(value: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def reduce_max(value: float, device=None) -> float:
    return _reduce(value, "max", device)


def reduce_sum(value: float, device=None) -> float:
    return _reduce(value, "sum", device)
