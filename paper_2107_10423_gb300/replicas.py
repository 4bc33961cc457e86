"""Whole-job throughput across ranks when every rank runs its own replica of the workload (one GPU per rank, no
data-path collective): the timed region ends when the slowest rank ends, and the work of all ranks counts."""
from __future__ import annotations


def aggregate(ms_local: float, units_local: float, device=None):
    """Returns (ms_max, units_total, units_per_s) over the default process group (or the local values if
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, units_local, units_local / (ms_local / 1e3)
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms, units = float(t.item()), float(u.item())
    return ms, units, units / (ms / 1e3)
