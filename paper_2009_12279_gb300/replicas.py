"""Replica parallelism for independent solves (one process per GPU).

The method's independent solves share nothing, so several GPUs run disjoint shares of
the request stream or replicas of a workload; the only communication is the timing and
count reduction at the end (max of the per-rank times, sum of the per-rank work).
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (every item goes to exactly one rank)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank / world size")
    return items[rank::world]


def reduce_timing(dist, elapsed_s: float, work: float, device=None):
    """(max elapsed over ranks, summed work over ranks) with torch.distributed `dist`;
    without a process group the local values are returned."""
    if dist is None or not dist.is_initialized():
        return elapsed_s, work
    import torch

    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())
