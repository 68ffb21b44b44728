"""Host-side logic of running independent replicas, one process per GPU.

The short-range force path has no exchange step within one system, so N GPUs
run N independent replicas of the same step (weak scaling).  What the ranks
share is only the measurement: a barrier around the timed region, the maximum
of the per-rank times, and the whole-job throughput = (units per rank x N) /
that time.  The process group comes from the usual torchrun environment
(RANK, LOCAL_RANK, WORLD_SIZE, MASTER_ADDR, MASTER_PORT).
"""

from __future__ import annotations

import os


def setup(backend: str = "nccl") -> tuple[int, int, int]:
    """(world size, rank, local rank); joins the process group when world > 1."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest value of x over the ranks (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_per_rank: float, ms_per_step: float, world: int, device: str = "cuda") -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    total = sum_over_ranks(units_per_rank, world, device)
    slowest = max_over_ranks(ms_per_step, world, device)
    return total / (slowest * 1e-3)
