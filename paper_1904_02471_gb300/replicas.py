"""Replica bookkeeping for runs on several GPUs of one node.

The CS and FD updates of independent lattices never exchange data, so the
multi-GPU form is replicas: every rank advances its own lattices and nothing
crosses ranks on the data path. Only the measurement is collective: ranks
meet at a barrier before and after the timed region, the job time is the
maximum over ranks, and the whole-job throughput counts every rank's work.
"""
from __future__ import annotations


def job_time(dist, t_local: float, device=None) -> float:
    """Maximum of the ranks' timed-region durations (t_local on one rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return t_local
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_job: float) -> float:
    """Units processed by all ranks per unit of job time (weak scaling: every
    rank processes units_per_rank)."""
    if t_job <= 0:
        raise ValueError("job time must be positive")
    return units_per_rank * world / t_job
