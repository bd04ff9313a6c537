"""Sharding of independent beams across ranks (one process per GPU).

Beams are independent problems (the paper's statistical realisations and test
beams), so they partition across GPUs with no collective in the data path:
each rank marches its own beams.  The only communication is the end-of-run
aggregation of timings and (optionally) results on the host.
"""
from __future__ import annotations


def partition(sizes: list, world: int) -> list:
    """Assign beam indices to `world` ranks: largest grid first, each to the
    rank with the fewest points so far (ties -> lowest rank).  Deterministic."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda b: (-int(sizes[b]) ** 2, b))
    load = [0] * world
    out = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(b)
        load[r] += int(sizes[b]) ** 2
    return [sorted(x) for x in out]


def my_beams(sizes: list, world: int, rank: int) -> list:
    return partition(sizes, world)[rank]


def aggregate(points_steps: float, ms: float, dist=None, device=None) -> tuple:
    """Whole-job throughput from per-rank work and time: sum of work over ranks
    divided by the slowest rank's time.  Returns (value per second, max ms).
    `device` holds the reduction tensors (a CUDA device for NCCL, CPU for gloo)."""
    if dist is None:
        return points_steps / (ms / 1e3), ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([points_steps], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(w.item()) / (float(t.item()) / 1e3), float(t.item())
