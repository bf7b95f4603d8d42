"""Row shards: the host side of a row-sharded run of the online DMD passes.

Sec. 2.3 costs the update at O(N r) per snapshot in matrix-vector products: every tall
pass is row-local and ends in a reduction of a few values (2 r0 + 3 for the projection and
residual pass, 2 for the credibility check, 1 for the norm of the first snapshot).  So the
rows split across GPUs, each GPU holding its rows of the basis and of the snapshots, and
the only exchange is that reduction.  To make the sharded result bitwise the unsharded one,
the rows are cut into B fixed row blocks (whole 64-row tiles, the same blocks the library's
kernels use, see odmd_get_row_blocks), each block's partial sums are computed the same way
wherever the block lives, and the per-block partials -- not per-shard sums -- are exchanged
(an all-gather) and added in block order on every rank.

This module holds that protocol for any torch.distributed process group (NCCL between GPUs,
gloo between CPU ranks).  On one GPU the library runs the same protocol through its
workspace (odmd_set_row_shards).
"""
from __future__ import annotations

from typing import Sequence

import numpy as np

TILE_ROWS = 64


def row_blocks(n: int, blocks: int) -> list[int]:
    """The blocks + 1 row boundaries: block b is 64-row tiles [b T / B, (b + 1) T / B)."""
    if n < 1 or blocks < 1:
        raise ValueError("n and blocks must be positive")
    tiles = (n + TILE_ROWS - 1) // TILE_ROWS
    if blocks > tiles:
        raise ValueError("more blocks than 64-row tiles")
    return [min(b * tiles // blocks * TILE_ROWS, n) for b in range(blocks + 1)]


def shard_blocks(blocks: int, shards: int, g: int) -> tuple[int, int]:
    """(first, count): shard g of `shards` holds the contiguous blocks [first, first + count)."""
    if not 1 <= shards <= blocks or not 0 <= g < shards:
        raise ValueError("need 1 <= shards <= blocks and 0 <= g < shards")
    first = g * blocks // shards
    return first, (g + 1) * blocks // shards - first


def exchange_partials(local, first: int, blocks: int, group=None):
    """All-gather of per-block partials: `local` is this rank's (count, nv) tensor for blocks
    [first, first + count); returns the (blocks, nv) tensor of every block, in block order, on
    every rank.  Ranks hold contiguous block ranges in rank order (shard_blocks)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    nv = local.shape[1]
    counts = [shard_blocks(blocks, world, g)[1] for g in range(world)]
    if local.shape[0] != counts[dist.get_rank(group)] or first != shard_blocks(blocks, world, dist.get_rank(group))[0]:
        raise ValueError("this rank's partials do not cover its shard of the blocks")
    width = max(counts)
    padded = torch.zeros((width, nv), dtype=local.dtype, device=local.device)
    padded[: local.shape[0]] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[:c] for p, c in zip(parts, counts)], dim=0)


def fold(partials: np.ndarray | Sequence[Sequence[float]]) -> np.ndarray:
    """The reduction of per-block partials: added one block after another, in block order."""
    p = np.asarray(partials, dtype=np.float64)
    out = np.zeros(p.shape[1], dtype=np.float64)
    for b in range(p.shape[0]):
        out = out + p[b]
    return out
