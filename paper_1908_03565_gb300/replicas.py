"""Multi-GPU bookkeeping for independent replicas.

The reconstruction shards by image (the draft's groups and frames decode
independently, 6.2 / 6.4), so N GPUs run N replicas with no exchange of
data: each rank reconstructs its own images, and the ranks only agree on
timing (a barrier around the timed region and the maximum time over ranks).
These helpers hold that host logic so it can be tested with the gloo
backend on CPU.
"""
import os


def rank_env():
    """(world_size, rank, local_rank) from the torchrun environment."""
    def get(k, d):
        try:
            return int(os.environ.get(k, d))
        except ValueError:
            return d
    return get("WORLD_SIZE", 1), get("RANK", 0), get("LOCAL_RANK", 0)


def shard(n_items, world, rank):
    """Indices of the items rank `rank` owns: a contiguous, balanced split
    (sizes differ by at most one)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value, dist=None, device="cpu"):
    """Largest `value` over all ranks (the job is as slow as its slowest
    replica)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_max, world):
    """Units per second of the whole job (weak scaling: every rank does
    `units_per_rank`)."""
    return world * units_per_rank / seconds_max
