"""One hull sharded across ranks (one process per GPU).

The hull of a union is the hull of the union of its parts' hulls: every
vertex of hull(S) is a vertex of the hull of the part that holds it, and
every vertex of a part's hull is a point of S (the same fact that makes
any polygon spanned by input points an exact filter, Section 2.2.2).  So
each rank computes the hull of its contiguous shard of the input with the
single-GPU pipeline (Section 2.1 steps 1-8), the ranks all-gather their
vertices (coordinates and global indices, padded to the largest count),
and the hull of the gathered vertices, again with the pipeline, is the
hull of the whole input.

Ties: the pipeline reports the smallest index among duplicate points.
Each shard's vertices are put in increasing global index before the
gather and the shards are concatenated in rank order (contiguous shards,
so rank order is index order), which keeps that rule across shards: the
hull of the union reports, for a point held by several shards, its
smallest global index.

The hull functions default to the CUDA pipeline (hull.Context.compute);
they can be replaced, for instance by a CPU routine to exercise the gather
and merge logic on ranks without a GPU.
"""
from __future__ import annotations

import numpy as np


def _default_hull(ctx):
    import torch

    def run(pts: np.ndarray) -> np.ndarray:
        if len(pts) == 0:
            return np.zeros(0, np.int64)
        t = torch.as_tensor(np.ascontiguousarray(pts, dtype=np.int32)).cuda(ctx.device)
        return ctx.compute(t).cpu().numpy().astype(np.int64)

    return run


def local_vertices(pts: np.ndarray, offset: int, hull_fn) -> tuple[np.ndarray, np.ndarray]:
    """Vertices of one shard's hull in increasing global index: (coordinates
    int32 (h, 2), global indices int64 (h,))."""
    pts = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 2))
    loc = np.sort(np.asarray(hull_fn(pts), dtype=np.int64))
    return pts[loc], loc + int(offset)


def merge(parts, hull_fn) -> np.ndarray:
    """Hull of the union of the shards' vertex sets `parts` (a list, in rank
    order, of (coordinates, global indices) as local_vertices returns):
    CCW global indices from the lexicographic minimum."""
    xy = np.concatenate([p[0] for p in parts], axis=0) if parts else np.zeros((0, 2), np.int32)
    gi = np.concatenate([p[1] for p in parts], axis=0) if parts else np.zeros(0, np.int64)
    if len(xy) == 0:
        return np.zeros(0, np.int64)
    h = np.asarray(hull_fn(xy), dtype=np.int64)
    return gi[h]


def gather_vertices(xy: np.ndarray, gi: np.ndarray, group=None, device=None):
    """All-gather of every rank's vertices over torch.distributed: the
    counts first, then the coordinates and indices padded to the largest
    count.  Returns the list of (coordinates, global indices) in rank
    order.  `device`: where the collective's tensors live (a CUDA device for
    NCCL, None for CPU backends such as gloo)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    dev = torch.device("cpu") if device is None else torch.device(device)
    cnt = torch.tensor([len(xy)], dtype=torch.int64, device=dev)
    counts = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(counts, cnt, group=group)
    counts = [int(c.item()) for c in counts]
    hmax = max(max(counts), 1)
    pxy = torch.zeros((hmax, 2), dtype=torch.int32, device=dev)
    pgi = torch.full((hmax,), -1, dtype=torch.int64, device=dev)
    if len(xy):
        pxy[: len(xy)] = torch.as_tensor(np.ascontiguousarray(xy, dtype=np.int32))
        pgi[: len(gi)] = torch.as_tensor(np.asarray(gi, dtype=np.int64))
    all_xy = [torch.empty_like(pxy) for _ in range(world)]
    all_gi = [torch.empty_like(pgi) for _ in range(world)]
    dist.all_gather(all_xy, pxy, group=group)
    dist.all_gather(all_gi, pgi, group=group)
    return [(all_xy[r][: counts[r]].cpu().numpy(), all_gi[r][: counts[r]].cpu().numpy()) for r in range(world)]


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous shard [lo, hi) of rank `rank` among `world` for n points."""
    return n * rank // world, n * (rank + 1) // world


def sharded_hull(pts_local: np.ndarray, offset: int, ctx=None, group=None, device=None,
                 hull_fn=None) -> np.ndarray:
    """Hull of the union of every rank's shard.  pts_local: this rank's
    contiguous shard (int32 (m, 2)); offset: the global index of its first
    point.  Every rank returns the same CCW global indices.  hull_fn (a
    function from an (m, 2) int32 array to hull indices) defaults to the
    CUDA pipeline of `ctx`."""
    if hull_fn is None:
        if ctx is None:
            raise ValueError("sharded_hull needs a hull.Context or a hull function")
        hull_fn = _default_hull(ctx)
    xy, gi = local_vertices(pts_local, offset, hull_fn)
    parts = gather_vertices(xy, gi, group=group, device=device)
    return merge(parts, hull_fn)
