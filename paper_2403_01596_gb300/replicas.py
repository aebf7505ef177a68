"""Independent replicas across ranks (one process per GPU).

The P2P operator of one point set has no exchange step when every box set
lives on one GPU, so a multi-GPU run is N independent replicas.  The only
cross-rank communication is timing: a barrier around the timed region and the
maximum of the per-rank times, so the whole-job throughput is
N x (per-replica work) / (slowest replica's time).
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(rank, local rank, world size) from the torchrun environment (1 process if absent)."""
    def env(name, default):
        try:
            return int(os.environ.get(name, default))
        except ValueError:
            return default
    return env("RANK", 0), env("LOCAL_RANK", 0), env("WORLD_SIZE", 1)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks of the default process group (the value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def job_throughput(units_per_replica: float, world_size: int, slowest_seconds: float) -> float:
    """Whole-job rate: every replica processes `units_per_replica` in at most `slowest_seconds`."""
    if slowest_seconds <= 0:
        raise ValueError("time must be positive")
    return world_size * units_per_replica / slowest_seconds
