"""Multi-GPU runs as independent replicas.

The method's domains are independent (the paper's runs are single-GPU and
have no exchange step), so N GPUs run N replicas of a workload with no
collective on the data path.  The only communication is the timing rule of
a multi-process run: every rank measures its own time, the job time is the
maximum over ranks, and the job throughput counts the work of all ranks.
"""
from __future__ import annotations


def job_throughput(local_seconds: float, local_units: float, group=None):
    """(units of all ranks / max over ranks of the time, max time, world size).
    Uses torch.distributed when it is initialised, else this process alone."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_units / local_seconds, local_seconds, 1
    world = dist.get_world_size(group)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()) / float(t.item()), float(t.item()), world
