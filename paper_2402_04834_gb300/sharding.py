"""Weak-scaling layout of a decoding job over several GPUs (one process each).

Syndromes are independent (Algorithm 1 decodes one syndrome at a time), so
the job shards by shot range with no exchange on the data path; the only
collective is the reduction of the timing (the slowest rank decides) and,
optionally, of the counters a Monte-Carlo run reports.
"""

from __future__ import annotations


def shot_range(rank: int, world: int, per_rank: int, first_shot: int = 0):
    """[start, stop) of the shots rank ``rank`` decodes; ranks never overlap."""
    if not (0 <= rank < world) or per_rank < 0:
        raise ValueError("bad rank / world / per_rank")
    start = first_shot + rank * per_rank
    return start, start + per_rank


def reduce_max(value: float, dist=None, device=None) -> float:
    """Maximum of ``value`` over all ranks (the job's wall time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, dist=None, device=None) -> float:
    """Sum of ``value`` over all ranks (e.g. failures, shots)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
