"""Replica bookkeeping for multi-GPU runs.

A single problem has no data-parallel split without per-level exchanges, so
several GPUs run independent replicas (one problem per rank) and the job's
throughput is all ranks' unknowns over the slowest rank's time.  These
helpers hold that arithmetic and the max-over-ranks reduction; they work with
any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput in millions of units per second."""
    return units_per_rank * world / (max_ms * 1e-3) / 1e6
