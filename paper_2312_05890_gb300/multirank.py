"""Runs over several GPUs of one node, one process per GPU (host side only).

The count partitions, it does not exchange.  Weak scaling: every rank counts
a problem of its own (rank r takes the workload's seed + r).  Strong
scaling: the ranks share one count, rank r taking shard r of the tree (the
`shard_*` options: every N-th subtree below a level g), and the whole count's
bracket is the sum of the shards' brackets (`sum_counts`).  Either way the
only collectives are the barriers around a timed region and the reductions
of its timings, unit counts and the two volume counters at the end.
"""
from __future__ import annotations

import os


def rank_env():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def weak_seed(seed: int, rank: int) -> int:
    """Seed of the problem rank `rank` counts: same shape, its own draw."""
    return seed + rank


def init(world: int):
    """torch.distributed for world > 1 (NCCL with GPUs, else gloo), or None."""
    if world <= 1:
        return None
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist


def barrier(dist) -> None:
    if dist is not None:
        dist.barrier()


def job_rate(local_ms: float, local_units: float, dist=None):
    """(max_ms, total_units, units per second) of the whole job."""
    import torch
    dev = "cpu"
    if dist is not None and dist.get_backend() == "nccl":
        dev = "cuda"
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    max_ms = float(t.item())
    total = float(u.item())
    return max_ms, total, total / (max_ms / 1e3)


def sum_counts(unsafe_lo: int, unsafe_hi: int, dist=None):
    """The whole count's bracket from the shards' (unsafe_lo, unsafe_hi): sums."""
    import torch
    dev = "cuda" if dist is not None and dist.get_backend() == "nccl" else "cpu"
    v = torch.tensor([int(unsafe_lo), int(unsafe_hi)], dtype=torch.int64, device=dev)
    if dist is not None:
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return int(v[0].item()), int(v[1].item())


def finish(dist) -> None:
    if dist is not None:
        dist.destroy_process_group()
