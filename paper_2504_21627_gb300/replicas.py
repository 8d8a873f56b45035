"""Replica aggregation for multi-GPU runs of the query.

The query shards trivially: rays are independent, so N GPUs run N replicas
of the same workload with no data-path collective. The only cross-rank step
is the measurement: the job's time is the slowest rank's, and its throughput
counts every rank's rays.
"""
from __future__ import annotations


def aggregate(ms_local: float, rays_local: int, group=None) -> tuple[float, int, float]:
    """(max over ranks of ms, total rays over ranks, Mrays/s of the job)."""
    import torch
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        r = torch.tensor([rays_local], dtype=torch.float64, device=dev)
        dist.all_reduce(r, op=dist.ReduceOp.SUM, group=group)
        ms, rays = float(t.item()), int(r.item())
    else:
        ms, rays = float(ms_local), int(rays_local)
    return ms, rays, rays / (ms / 1e3) / 1e6


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n independent rays for one rank (used
    when a fixed batch is split instead of replicated)."""
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)
