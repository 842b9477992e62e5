"""Host-side logic for running the particle path on several GPUs, one process each.

The path splits into independent units with no exchange between them: the
members of an ensemble (independent meshes and particle sets) or whole
replicas of one problem.  A rank advances its own units with the same
library calls as a single GPU; the only collectives are the two reductions
of the timing protocol (maximum elapsed time, summed work), outside the
data path.

Assigning ensemble members to ranks is the balancing problem the paper
discusses for particles per process (Sec. 2.5, load balancing): the members
are weighted by their particle counts and dealt out by the longest-
processing-time rule, which keeps the heaviest rank within 4/3 of the best
possible split.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment; (0, 1, 0) without one."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def partition_by_weight(weights, world: int) -> list[list[int]]:
    """Deal unit indices out to `world` ranks by the longest-processing-time rule.

    Units are taken heaviest first (ties: lower index first) and each goes to
    the rank with the smallest load so far (ties: lower rank).  Every index
    appears in exactly one list; each list is returned in increasing index
    order so that a rank advances its members in their global order.  The
    result depends on the weights alone, so every rank computes the same split
    without communicating.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [int(v) for v in weights]
    if any(v < 0 for v in w):
        raise ValueError("weights must be non-negative")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += w[i]
    return [sorted(p) for p in parts]


def reduce_timing(elapsed, units, device=None, group=None) -> tuple[list[float], list[float]]:
    """Timing protocol over ranks: the maximum of each elapsed time and the sum of each work count.

    elapsed, units: sequences of floats measured on this rank.  With one
    process (no initialised process group) they are returned unchanged.
    `device` is where the reduction tensors live (a CUDA device for NCCL,
    None = CPU for gloo).
    """
    import torch
    import torch.distributed as dist

    elapsed = [float(v) for v in elapsed]
    units = [float(v) for v in units]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return elapsed, units
    t = torch.tensor(elapsed, dtype=torch.float64, device=device)
    u = torch.tensor(units, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.cpu()], [float(v) for v in u.cpu()]
