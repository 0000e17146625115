"""Host-side multi-process helpers.

Targets of a network are independent (Supporting Information, Run-time on CPU
and GPU: one computing node per target), so several processes, one per GPU,
split them without exchanging any data on the compute path; only the final
per-target results and timing are gathered on the host.
"""
from __future__ import annotations


def shard_targets(n_proc: int, rank: int, world: int) -> list:
    """Round-robin split of targets 0..n_proc-1 over `world` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, n_proc, world))


def combine_timing(dist, times_ms, counts, device="cpu"):
    """Max over ranks of each time and sum over ranks of each count (every
    rank gets the result).  `dist` is torch.distributed or None (one rank)."""
    import torch
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def gather_results(dist, obj):
    """All ranks' Python objects, in rank order (one rank: [obj])."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
