"""Points across GPUs: each rank renders a contiguous shard of the scene (a Scene with the
shard's index_base), the key images are combined by one minimum across ranks, and each rank
resolves the pixels its own points won; the resolved planes add up across ranks.

Sec. 3.2's render pass keeps, per pixel, the minimum key over all points; a minimum of the
shards' minima is the same key, bit for bit, because every key carries its global index.  The
only exchange is that minimum (8 bytes per pixel) and the sum of the resolved planes (every
pixel has one owner, the others contribute zeros).  Collectives go through torch.distributed;
the arithmetic on the keys (the sign flip that turns their unsigned order into int64 order, so a
signed MIN collective combines them) runs in the library.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import nrv


def shard_range(n: int, rank: int, world: int):
    """Contiguous index range [lo, hi) of rank's shard of n points."""
    return n * rank // world, n * (rank + 1) // world


def combine_keys_(keys, group=None, flip=None):
    """In place: keys (int64 tensor holding uint64 keys) becomes the minimum over all ranks."""
    flip = nrv.keys_flip_sign if flip is None else flip
    flip(keys)
    dist.all_reduce(keys, op=dist.ReduceOp.MIN, group=group)
    flip(keys)


def combine_planes_(planes, group=None):
    """In place: every resolved plane (depth bits, coverage, attribute words) becomes the sum
    over ranks, i.e. the owner's value."""
    for p in planes:
        if p is not None:
            dist.all_reduce(p, op=dist.ReduceOp.SUM, group=group)


def render_split(scene: nrv.Scene, view, key, depth=None, mask=None, gattr=None, group=None,
                 stream=None):
    """Render this rank's shard, combine the key image across ranks, resolve the pixels this
    shard owns and add the planes across ranks: on return every rank holds the whole scene's
    G-buffer of `view`."""
    nrv.rasterize(scene, [view], [key], stream=stream)
    combine_keys_(key, group)
    nrv.resolve(scene, view, key, depth, mask, gattr, stream=stream)
    combine_planes_([depth, mask, gattr], group)
