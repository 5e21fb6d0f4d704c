"""Independent problems over ranks (one process per GPU), and the whole-job
rate of a timed region.

The slices of one structure form a serial chain, so one structure is never
split between GPUs. What shards are independent units: separate volumes,
the structures of a batch, and training samples. They are partitioned by
index and exchange nothing on the data path. The only collectives are on the
timing: the maximum of the ranks' times and the sum of their units.
"""
from __future__ import annotations


def shard(n, rank, world):
    """The contiguous block of range(n) that `rank` of `world` owns.

    The blocks are balanced: the first n % world ranks take one unit more.
    Over all ranks they are disjoint and cover range(n). A rank past the end
    gets an empty range."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("shard: need 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def whole_job_rate(units_local, ms_local, device=None):
    """Return (rate, ms) for the whole job.

    rate is the units of all ranks divided by the slowest rank's time, in
    units per second. ms is that slowest time. Without an initialised
    process group, or with a group of one, these are the local figures."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units_local / (ms_local / 1e3), float(ms_local)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) / 1e3), float(t.item())
