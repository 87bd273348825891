"""Rank bookkeeping for runs on several GPUs of one node (one process per GPU).

The framed blocks are independent problems, so a multi-GPU run shards work by
giving every rank its own batch (weak scaling); the only collectives are the
timing barrier and the maximum of the per-rank times, never on the data path.
"""

import os


def rank_info():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def batch_seed(seed, rank):
    """Seed of a rank's own right-hand sides (distinct per rank)."""
    return seed + 1000 * rank


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value, world, device=None):
    """Largest per-rank value (e.g. the time of the timed region)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest time."""
    return world * units_per_rank / seconds
