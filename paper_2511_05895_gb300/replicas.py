"""Multi-GPU runs as independent replicas.

The dynamic max-flow path has no exchange step (every push-relabel round
does fine-grained atomics on arbitrary neighbours and the BFS is global), so
N GPUs run N independent graphs, one per rank, with no collective on the data
path.  Only the benchmark's bookkeeping crosses ranks: a barrier before the
timed region and the maximum of the per-rank times after it.
"""
from __future__ import annotations

import os


def rank_world():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, seconds_this_rank: float, device=None) -> float:
    """Units of all ranks per second, timed by the slowest rank (weak scaling:
    every rank processes the same number of units)."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return world * units_per_rank / max_over_ranks(seconds_this_rank, device)
