"""Replicas over several GPUs of one node.

The executor does not shard a nest over GPUs: every GPU runs its own copy of
the workload (weak scaling), and the ranks only agree on time.  The whole-job
throughput is the units all ranks processed over the slowest rank's time.
These helpers work with any initialised torch.distributed process group
(NCCL on GPUs; gloo on CPUs in the tests) and with a single process."""
from __future__ import annotations


def world() -> tuple[int, int]:
    """(world size, rank) of the default process group, (1, 0) without one."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_world_size(), dist.get_rank()
    return 1, 0


def barrier() -> None:
    import torch.distributed as dist
    if world()[0] > 1:
        dist.barrier()


def max_over_ranks(value: float, device="cpu") -> float:
    """The largest `value` over all ranks (every rank gets it)."""
    import torch
    import torch.distributed as dist
    if world()[0] == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, seconds: float, device="cpu") -> tuple[float, float]:
    """(units of all ranks per second of the slowest rank, that rank's seconds)."""
    ws = world()[0]
    slowest = max_over_ranks(seconds, device)
    return units_per_rank * ws / slowest, slowest
