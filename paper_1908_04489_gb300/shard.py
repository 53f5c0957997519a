"""One instance's sweep split over the ranks of a process group.

For a fixed controller the u0 step of every x0 point is independent of the
others (the parallelism of the paper's Section IV-A), so each rank holds the
same instance, searches a contiguous range of x0 points (``ucp_sweep_part``),
the ranges' new values are all-gathered, and every rank finishes the sweep on
the whole new controller (``ucp_sweep_finish``: u1 step, tables, J).  The
u1 step and J are repeated on every rank, so every rank holds the same
state, bit for bit equal to one process sweeping alone.

This module only moves the values between the library and
``torch.distributed``; every step of the sweep runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np


def x_ranges(n_x: int, world: int):
    """Contiguous ranges [lo, hi) of the x0 points, one per rank, sizes
    differing by at most one (rank r gets the r-th)."""
    base, extra = divmod(int(n_x), int(world))
    out, lo = [], 0
    for r in range(int(world)):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def sweep(inst, n: int = 1, group=None):
    """n sweeps of `inst`, split over the ranks of `group` (the default
    group if None).  `inst` needs n_x, sweep_part(i0, i1) and
    sweep_finish(f); the exchange uses CPU tensors with gloo and device
    tensors with NCCL."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    ranges = x_ranges(inst.n_x, world)
    lo, hi = ranges[rank]
    width = max(h - l for l, h in ranges)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    for _ in range(int(n)):
        part = inst.sweep_part(lo, hi)
        buf = torch.zeros(width, dtype=torch.float64)
        buf[:hi - lo] = torch.from_numpy(np.ascontiguousarray(part))
        buf = buf.to(dev)
        parts = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(parts, buf, group=group)
        f = np.concatenate([parts[r][:ranges[r][1] - ranges[r][0]].cpu().numpy()
                            for r in range(world)])
        inst.sweep_finish(f)
