"""One G0W0 job split across ranks (one process and one GPU per rank).

The library partitions the work itself (gw_set_shard): each rank builds the imaginary-axis table for its block of
frequency positions and solves every world-th residue right-hand side; the only exchanges are two element-wise
sums of host arrays, the W table once per build and the per-target residue sums (R, dR/domega) once per Sigma
evaluation.  This module supplies the sum as a C callback over torch.distributed (gloo sums host tensors in place;
NCCL sums a device copy)."""
from __future__ import annotations

import ctypes

import numpy as np

ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_longlong, ctypes.c_void_p)


def make_allreduce(group=None, device=None):
    """A gw_allreduce_fn that sums buf[n] over the ranks of ``group`` (default: the default process group).
    ``device``: a CUDA device for NCCL groups (the buffer is copied there and back); None sums in host memory."""
    import torch
    import torch.distributed as dist

    def cb(buf, n, ctx):
        try:
            a = np.ctypeslib.as_array(buf, shape=(int(n),))
            t = torch.from_numpy(a)
            if device is not None:
                d = t.to(device)
                dist.all_reduce(d, op=dist.ReduceOp.SUM, group=group)
                t.copy_(d.cpu())
            else:
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return 0
        except Exception:
            return 1

    return ALLREDUCE_FN(cb)


def shard_columns(n_freq: int, rank: int, world: int):
    """The block [p0, p1) of frequency positions a rank computes (the library's partition; host only)."""
    from . import gw
    p0, p1 = ctypes.c_int(), ctypes.c_int()
    st = gw.load().gw_shard_columns(int(n_freq), int(rank), int(world), ctypes.byref(p0), ctypes.byref(p1))
    if st != gw.GW_OK:
        raise gw.GWError(st, "gw_shard_columns")
    return p0.value, p1.value


def position_column(p: int, n_freq: int) -> int:
    """W-table column of frequency position p (position 0 is xi = 0, stored last)."""
    return n_freq if p == 0 else p - 1


def owns_residue(j: int, rank: int, world: int) -> bool:
    """Right-hand side j of a Sigma evaluation's residue list belongs to rank j % world."""
    return j % world == rank
