"""Replica bookkeeping for `bench.py --gpus N` (one process per GPU, launched
by torch.distributed.run): each rank solves its own copy of the workload, no
data-path collective; only the timing is combined.

  dist_env()                      RANK, WORLD_SIZE, LOCAL_RANK from the environment
  max_over_ranks(x, device)       the slowest rank's time (all_reduce MAX), x itself for one rank
  job_throughput(ms, world)       whole-job ground states per second: world solves in ms
"""
from __future__ import annotations

import os


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device=None) -> float:
    """Max of x over the ranks of the default process group (any backend:
    NCCL with a CUDA device, gloo on the CPU); x when there is no group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_per_step: float, world: int) -> float:
    """Each of the `world` replicas solves one instance per step; the step time
    is the slowest replica's, so the job delivers world instances per step."""
    return world * 1000.0 / ms_per_step
