"""Multi-GPU sharding of a batch (one process per GPU).

Element integration has no communication between elements (Sec. 2: every
element matrix depends only on its own geometry and coefficients), so a
batch splits into contiguous element ranges, one per rank, and each rank
integrates its range with no collective at all.  Ranges are balanced by
the algorithmic work of their elements, F(p) = 8 N_sh^2 N_q + 2 N_sh N_q +
220 N_q, so a mixed-degree batch gives every rank about the same work.
``gather_outputs`` concatenates the ranks' results in element order, for
the case where one process wants the whole batch; it is not part of the
integration itself.

Pure host logic plus torch.distributed; it works with the gloo backend on
CPU tensors and with NCCL on CUDA tensors.
"""
from __future__ import annotations

import numpy as np


def element_flops(degrees) -> np.ndarray:
    """F(p) per element (int64) for an int array of degrees 1..7."""
    p = np.asarray(degrees, dtype=np.int64)
    s = (p + 1) * (p + 1) * (p + 2) // 2
    q = (p + 1) ** 3
    return 8 * s * s * q + 2 * s * q + 220 * q


def partition(degrees, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [start, end) of elements, one per rank, that split
    the prefix sum of F(p) at the multiples of total/world.  Every element
    belongs to exactly one range; ranges may be empty."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = element_flops(degrees)
    n = len(w)
    if n == 0:
        return [(0, 0)] * world
    c = np.cumsum(w)
    total = int(c[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        # c[k-1] < target <= c[k]: end the range after element k-1 or after
        # element k, whichever prefix sum is closer to the target
        k = int(np.searchsorted(c, target, side="left"))
        below = c[k - 1] if k > 0 else 0
        cut = k if k >= n or target - below <= c[k] - target else k + 1
        cuts.append(min(max(cut, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard(w: dict, rank: int, world: int) -> dict:
    """The slice of workload ``w`` (the dict of ``inputs.workload``) that
    rank ``rank`` integrates: geometry, coefficients (per element, or per
    point by the points of the range), degrees.  Adds ``start``/``end``."""
    degrees = w["degree"] if w.get("degree") is not None else np.full(len(w["geom"]), w["p"], dtype=np.int32)
    lo, hi = partition(degrees, world)[rank]
    out = dict(w)
    out["geom"] = np.ascontiguousarray(w["geom"][lo:hi])
    out["degree"] = np.ascontiguousarray(degrees[lo:hi])
    if w.get("per_qp"):
        q = (np.asarray(degrees, dtype=np.int64) + 1) ** 3
        qo = np.concatenate([[0], np.cumsum(q)])
        a, b = int(qo[lo]), int(qo[hi])
    else:
        a, b = lo, hi
    for k in ("K", "b", "c", "f"):
        out[k] = np.ascontiguousarray(w[k][a:b])
    out["start"], out["end"] = lo, hi
    return out


def gather_outputs(tensors, group=None):
    """All-gather 1-D tensors of different lengths (one per rank) and
    concatenate them in rank order on every rank.  ``tensors`` is a tuple of
    local tensors (A, b, status, ...); returns the tuple of concatenations."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    out = []
    for t in tensors:
        t = t.reshape(-1).contiguous()
        n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
        sizes = [torch.zeros_like(n) for _ in range(world)]
        dist.all_gather(sizes, n, group=group)
        sizes = [int(x.item()) for x in sizes]
        m = max(sizes) if sizes else 0
        pad = torch.zeros(m, dtype=t.dtype, device=t.device)
        pad[: t.numel()] = t
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        out.append(torch.cat([parts[r][: sizes[r]] for r in range(world)]))
    return tuple(out)
