"""Replicas over evaluation points: one model per GPU, points split across ranks.

The points of a batch (stencil, line-search or integration points) are
independent, which is the paper's "level 1" parallelism (Sec. 3.1): each rank
evaluates a contiguous shard of the batch on its own model replica and the
ranks exchange only the small per-point results (f, grad, status), never any
factorisation data.  Works with any torch.distributed backend (NCCL on GPUs,
gloo on CPUs).
"""
import numpy as np


def shard_bounds(n_points: int, rank: int, world: int):
    """[start, stop) of rank's contiguous share; shares differ by at most one point."""
    if not (0 <= rank < world) or n_points < 0:
        raise ValueError("bad rank / world / n_points")
    base, extra = divmod(n_points, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard(points, rank: int, world: int):
    s, e = shard_bounds(len(points), rank, world)
    return points[s:e]


def gather_results(local, n_points: int, group=None):
    """Concatenate every rank's per-point rows (numpy array [k, ...]) in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    local = np.ascontiguousarray(local, dtype=np.float64)
    width = int(np.prod(local.shape[1:])) if local.ndim > 1 else 1
    maxk = -(-n_points // world)
    buf = torch.zeros(maxk, width, dtype=torch.float64)
    buf[:local.shape[0]] = torch.from_numpy(local.reshape(local.shape[0], width))
    backend = dist.get_backend(group)
    if backend == "nccl":
        buf = buf.cuda()
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    rows = []
    for r, part in enumerate(parts):
        s, e = shard_bounds(n_points, r, world)
        rows.append(part[: e - s].cpu().numpy())
    out = np.concatenate(rows, 0)
    return out.reshape((n_points,) + local.shape[1:])


def max_over_ranks(value: float, group=None):
    """The largest of a scalar across ranks (e.g. the step time of the slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t[0])
