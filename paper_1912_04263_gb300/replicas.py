"""Replica bookkeeping for runs on several GPUs of one node.

The solver does not shard one problem across GPUs (the paper leaves
multi-GPU to future work; the path has no natural single exchange step).
Several GPUs run independent problems, one process per GPU: rank r solves
the instance with seed base + r, and the job's throughput is the number of
solves of all ranks divided by the slowest rank's time.  The only
collectives are a barrier around the timed region and a max-reduction of
the elapsed time; they run on whatever process group the caller created
(NCCL on GPUs, gloo on CPUs in the tests).
"""
from __future__ import annotations


def replica_seed(base_seed: int, rank: int) -> int:
    """Seed of the instance rank `rank` solves (distinct per rank)."""
    return int(base_seed) + int(rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """All-reduce MAX of one float over the process group (identity without
    one).  device: where the group's tensors live (a CUDA device for NCCL,
    None for gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_elapsed_s: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's
    time (weak scaling: per-rank work is fixed as the rank count grows)."""
    if max_elapsed_s <= 0.0:
        raise ValueError("elapsed time must be positive")
    return units_per_rank * world / max_elapsed_s
