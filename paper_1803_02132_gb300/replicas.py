"""Host side of independent replicas: one process per GPU, each measuring its own realisation.

Independent mocks or realisations share nothing on the data path (the multipoles of one
catalogue need only that catalogue), so several GPUs run whole measurements side by side.
Only timings and the small FP64 outputs cross processes, through torch.distributed (NCCL
between GPUs, gloo on CPU).
"""
from __future__ import annotations

import numpy as np


def _active(dist):
    return dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of a list of floats over all ranks: the slowest rank sets a step's time."""
    vals = [float(v) for v in values]
    if not _active(dist):
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def weak_scaling_rate(units_per_rank, ms_per_step, world):
    """Whole-job throughput: the units all ranks processed per second at the slowest rank's time."""
    return world * units_per_rank / (ms_per_step / 1e3)


def gather_outputs(out, dist=None, dst=0):
    """The output dicts (name -> FP64 array) of every rank, in rank order, on rank dst; None elsewhere."""
    if not _active(dist):
        return [out]
    objs = [None] * dist.get_world_size()
    dist.all_gather_object(objs, {k: np.asarray(v, dtype=np.float64) for k, v in out.items()})
    return objs if dist.get_rank() == dst else None
