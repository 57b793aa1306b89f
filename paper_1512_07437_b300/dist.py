"""Multi-GPU host logic: one process per GPU, independent work per rank.

The pairs of the posterior stage are independent and need no exchange, so
ranks share nothing on the data path (each processes its own families: weak
scaling).  They meet only to agree on timing: a barrier on both sides of the
timed region, the maximum of the per-rank times, and sums of the work done.
The process group is NCCL with GPUs, gloo on CPU.
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> bool:
    """Joins the process group when world_size > 1; returns whether it did."""
    import torch
    import torch.distributed as dist
    _, world, _ = env()
    if world <= 1 or dist.is_initialized():
        return dist.is_initialized()
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    dist.init_process_group(backend)
    return True


def _reduce(x: float, op) -> float:
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


def barrier():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()


def rank_seed(base: int, rank: int) -> int:
    """Seed of the synthetic workload of a rank (distinct per rank)."""
    return int(base) + 7919 * int(rank)


def whole_job_rate(units_this_rank: float, seconds_this_rank: float) -> float:
    """Units of all ranks over the slowest rank's time (units per second)."""
    units = sum_over_ranks(units_this_rank)
    secs = max_over_ranks(seconds_this_rank)
    return units / secs if secs > 0 else 0.0


def finalize():
    import torch.distributed as dist
    if dist.is_initialized():
        dist.destroy_process_group()
