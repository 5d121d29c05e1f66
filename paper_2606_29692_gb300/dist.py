"""Host-side helpers for running independent work on several GPUs.

The hot path has no exchange step: states, trajectories and requests are
independent, so each rank (one process per GPU) takes its own units and the
only collective is a reduction of timings.  Backend-agnostic: NCCL on GPUs,
gloo for the CPU tests of this logic.
"""

from __future__ import annotations

import os


def world_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend, device=None):
    """Join the process group when world_size > 1 (env:// rendezvous)."""
    import torch.distributed as dist
    rank, world, _ = world_info()
    if world > 1 and not dist.is_initialized():
        kw = {"device_id": device} if device is not None else {}
        dist.init_process_group(backend, **kw)
    return rank, world


def shard_range(n_units, rank, world):
    """Contiguous block [lo, hi) of n_units for `rank`; blocks tile 0..n_units."""
    base, rem = divmod(int(n_units), int(world))
    lo = rank * base + min(rank, rem)
    return lo, lo + base + (1 if rank < rem else 0)


def rank_seed(base_seed, rank):
    """Seed of a rank's own synthetic units (weak scaling: every rank draws
    a different, equally sized batch)."""
    return int(base_seed) + 7919 * int(rank)


def max_over_ranks(x, device="cpu"):
    """Maximum of a float over all ranks (the job's time is its slowest rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device="cpu"):
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def weak_scaling_value(units_per_rank, world, steps, t_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return float(units_per_rank) * int(world) * int(steps) / float(t_max)
