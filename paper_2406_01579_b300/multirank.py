"""Weak scaling over ranks, one GPU per rank.

The views of a training step are independent (each view's lists, blend and
record gradients are its own): each rank renders its own views of the scene.
The one exchange of the step is the sum of the scene's vertex gradients over
the ranks (dV, df, drgb: each rank's views give part of them), one
all-reduce per tensor after the backward.  The other collectives are the
barrier around the timed region and two reductions of the timing: the
slowest rank's time (max) and the pixels all ranks rendered (sum).  The job's
throughput is then the pixels of all ranks over the slowest rank's time.
"""

from __future__ import annotations

import numpy as np


def rank_cameras(base_cams, rank: int, width: int, height: int, seed: int = 1000):
    """The cameras rank ``rank`` renders: the workload's own for rank 0, the
    same number of random cameras (seeded by the rank) for the others."""
    if rank == 0:
        return list(base_cams)
    from .camera import on_sphere
    rng = np.random.default_rng(seed + rank)
    return [on_sphere(rng, width, height) for _ in range(len(base_cams))]


def job_mpix_s(local_pixels_per_step: int, steps: int, local_elapsed_s: float, dist=None,
               device=None) -> float:
    """Throughput of the whole job in Mpixel/s: the pixels all ranks rendered
    in ``steps`` steps over the slowest rank's time.  ``dist`` is
    torch.distributed (None: one rank); ``device`` the tensor device of its
    backend (cuda for NCCL, cpu for gloo)."""
    pixels, elapsed = float(local_pixels_per_step), float(local_elapsed_s)
    if dist is not None:
        import torch
        p = torch.tensor([pixels], dtype=torch.float64, device=device)
        t = torch.tensor([elapsed], dtype=torch.float64, device=device)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        pixels, elapsed = float(p.item()), float(t.item())
    return pixels * steps / elapsed / 1e6


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest of the ranks' values of x (x itself with one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_grads(grads, dist=None) -> None:
    """Sum each scene's vertex gradients (dV, df, drgb) over the ranks, in
    place: afterwards every rank holds the gradient of all ranks' views."""
    if dist is None:
        return
    for g in grads:
        for t in g:
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
