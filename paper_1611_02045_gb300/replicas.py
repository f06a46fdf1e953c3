"""Replica bookkeeping for `bench.py --gpus N` (one process per GPU, launched
by torch.distributed.run): each rank solves its own copy of the workload, no
data-path collective; only the timing is combined.

  dist_env()                      RANK, WORLD_SIZE, LOCAL_RANK from the environment
  max_over_ranks(x, device)       the slowest rank's time (all_reduce MAX), x itself for one rank
  job_throughput(ms, world)       whole-job ground states per second: world solves in ms
  instance_share(count, r, world) the independent instances rank r solves (index = r mod world)
  sum_over_ranks(values, device)  host-side totals of per-rank report counts (all_reduce SUM)
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


def instance_share(count: int, rank: int, world: int) -> list:
    """Indices of the independent instances (of `count`) that rank `rank` of
    `world` solves: those with index = rank (mod world).  The shares are
    disjoint, cover every instance, and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    return list(range(rank, count, world))


def sum_over_ranks(values, device=None):
    """Element-wise sum of a list of numbers over the ranks of the default
    process group (report counts gathered on the host); the list itself when
    there is no group."""
    import torch
    import torch.distributed as dist
    vals = [float(v) for v in values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return vals
    t = torch.tensor(vals, dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t)
    return [float(v) for v in t.tolist()]
