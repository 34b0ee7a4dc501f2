"""Host-side helpers for running the coupling benchmark on several GPUs of
one node: one process per GPU (``torchrun``), each stepping its own
independent box or boxes — the workload shards by whole boxes, so there is
no data-path collective (weak scaling); only the timing is reduced (the
slowest rank sets the time)."""

from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def box_seed(base, rank):
    """Seed of this rank's box: every rank draws an independent box."""
    return int(base) + int(rank)


def batched_seed0(rank, nbox=64):
    """First seed of this rank's batch of boxes (ranks get disjoint seeds)."""
    return int(nbox) * int(rank)


def max_over_ranks(value, device=None):
    """The largest value over the ranks of the default process group (the
    value itself when there is no group or a single rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processed units_per_rank in at most
    `seconds`."""
    return float(world) * float(units_per_rank) / float(seconds)
