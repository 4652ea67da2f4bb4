"""Multi-process sharding of the ray-tracing work (no collective on the data path).

Rays are independent, so a job splits into disjoint pieces with no exchange step:
either whole cameras (an inclination sweep, one camera per rank) or contiguous pixel
ranges of one camera (traced with gt_trace_range).  The only collectives are the
timing barrier and the max/sum reductions of the benchmark's timings.
"""
from __future__ import annotations

import dataclasses
import math


def sweep_camera(cam, rank: int, world: int, step_deg: float = 1.0):
    """Camera of `rank` in an inclination sweep: theta0 - rank * step_deg (degrees)."""
    if world <= 1:
        return cam
    return dataclasses.replace(cam, theta0=cam.theta0 - rank * step_deg * math.pi / 180.0)


def pixel_range(n_rays: int, rank: int, world: int):
    """Contiguous [first, first + count) share of n_rays for `rank` (sizes differ by <= 1)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_rays, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def reduce_timing(dist, seconds: float, units: float, device=None):
    """Job time = max over ranks, job units = sum over ranks (torch.distributed)."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
