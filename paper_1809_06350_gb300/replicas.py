"""Replica runs on several GPUs of one node (one process per GPU, torch.distributed).

The Newton step of one mesh is not sharded: each rank solves its own copy
(same workload per rank), so a multi-GPU run needs only a barrier around the
timed region and two host-side reductions of the results: the job's time is
the slowest rank's, its work the sum over ranks. No collective runs inside
the solve.
"""
from __future__ import annotations


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def reduce_timing(ms: float, work: int, device="cpu") -> tuple[float, int]:
    """(max over ranks of ms, sum over ranks of work); identity on one rank.
    `device` is where the two scalars travel (a CUDA device for NCCL, the CPU
    for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), int(work)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(w.item()))
