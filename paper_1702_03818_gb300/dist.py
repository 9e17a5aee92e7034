"""Host-side multi-rank helpers (one process per GPU, launched by torchrun).

The stage loop itself has no exchange step: a single grid would need a halo exchange to be
split (not built), and independent problems (the batched workload) are simply divided among
ranks.  These helpers do the division and the timing reductions; they run on any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations


def shard_indices(n_items: int, rank: int, world: int) -> list:
    """Items of this rank: i = rank, rank + world, ... (round-robin, no item twice)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, n_items, world))


def _reduce(x: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    return _reduce(x, "max", device)


def sum_over_ranks(x: float, device=None) -> float:
    """The sum over all ranks (the whole job's work)."""
    return _reduce(x, "sum", device)


def barrier(device=None) -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        if device is not None and getattr(device, "type", "cpu") == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()
