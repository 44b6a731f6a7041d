"""Tile sharding of the blend across ranks (one process per GPU).

Tiles are independent, so rank r of N blends only the global tiles
t = r, r + N, r + 2N, ... (the library's shard_count / shard_index options;
the kernels map their queue item q to tile q * N + r).  The forward pass
needs no exchange: each rank holds its tiles' pixels.  The backward pass adds
each rank's tiles' contributions to the per-Gaussian gradients, so one
all-reduce (sum) of those buffers gives every rank the full gradient — the
only collective on the path.
"""
from __future__ import annotations

import torch

from . import gs


def shard_tiles(total_tiles: int, rank: int, world: int) -> list[int]:
    """Global tile ids blended by `rank` of `world` (the kernels' partition)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of world {world}")
    return list(range(rank, total_tiles, world))


def allreduce_gradients(grads: dict, group=None) -> dict:
    """Sum each gradient buffer over the ranks of `group`, in place."""
    import torch.distributed as dist
    for t in grads.values():
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return grads


def blend_step_sharded(width: int, height: int, bs: dict, proj: dict, opacity: torch.Tensor, variant: str,
                       dL_dimage: torch.Tensor, rank: int, world: int, bg=(0.0, 0.0, 0.0), group=None,
                       gather_image: bool = False, reduce: bool = True) -> tuple[dict, dict]:
    """Forward and backward blend of this rank's tiles, then the gradient
    all-reduce.  Every rank must hold the same projection and sorted lists
    (each runs gs_project and gs_bin_sort itself, or receives them).  With
    gather_image the image, T_final and n_contrib are summed too (each pixel
    is written by exactly one rank, the rest are zero).  reduce=False skips
    the collectives (the caller sums the shards itself)."""
    opts = gs.make_opts(variant, bg=bg, shard_count=world, shard_index=rank)
    fwd = gs.blend_forward(width, height, bs, proj, opacity, opts)
    grads = gs.blend_backward(width, height, bs, proj, opacity, opts, fwd, dL_dimage)
    if world > 1 and reduce:
        allreduce_gradients(grads, group)
        if gather_image:
            import torch.distributed as dist
            for t in fwd.values():
                dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return fwd, grads
