"""Host logic of multi-GPU runs.  Trials and instances are independent
(Section III), so a job on N GPUs is N replicas of the workload, one process
per GPU, each with its own seeds: no collective on the data path.  The only
exchanges are timing (the slowest rank's step time, taken as the job's) and,
for statistics over the whole job, a gather of every rank's final cuts.

Works with any torch.distributed backend: NCCL with CUDA tensors on GPUs,
gloo with CPU tensors (how the tests run it on the CPU).
"""
from __future__ import annotations

import os

SEED_STRIDE = 1_000_003


def env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int, step: int) -> int:
    """Seed of one replica's step: distinct across ranks and steps."""
    return int(base) + SEED_STRIDE * int(rank) + int(step)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over the ranks (the slowest rank's time); the value
    itself without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds


def gather_cuts(cuts, dist=None):
    """Every rank's final cuts concatenated in rank order (the statistics of
    Eq. 3-5 over the whole job); the rank's own cuts without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return cuts
    import torch
    parts = [torch.empty_like(cuts) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, cuts)
    return torch.cat(parts)
