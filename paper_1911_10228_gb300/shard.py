"""Sharding one solve over several GPUs by target blocks (multi-GPU form of the
paper's distribution of octants over processes, Sec. 4).

Every rank holds the whole source (the input is replicated; on GB300-class
memory a 512^3-equivalent FP32 source is well under 1 GB) and creates a block
set that wants only its own targets (``flgf_blockset_create_masked``): the
spectrum products, inverse FFTs and the downward pass then run for those
targets and their octree ancestors only, so the dominant work splits across
the ranks and the solve itself needs no exchange.  Owned blocks are
contiguous chunks of the Morton (Z-order) curve of each level, of nearly equal
size, so a rank's targets are spatially compact and the blocks whose sources
it transforms redundantly (its halo) stay a thin layer.  The ranks gather
their owned blocks afterwards if one of them needs the whole field.
"""
from __future__ import annotations

import numpy as np


def morton_keys(coords) -> np.ndarray:
    """Z-order key of every block (coordinates shifted to start at 0, 21 bits per axis)."""
    c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
    if c.size == 0:
        return np.zeros(0, dtype=np.uint64)
    c = (c - c.min(axis=0)).astype(np.uint64)
    key = np.zeros(c.shape[0], dtype=np.uint64)
    for bit in range(21):
        for a in range(3):
            key |= ((c[:, a] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(3 * bit + (2 - a))
    return key


def morton_partition(coords, n_parts: int) -> np.ndarray:
    """Owner (0..n_parts-1) of every block: contiguous Morton-order chunks whose
    sizes differ by at most one."""
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    keys = morton_keys(coords)
    order = np.argsort(keys, kind="stable")
    owner = np.empty(keys.size, dtype=np.int64)
    bounds = np.linspace(0, keys.size, n_parts + 1).round().astype(np.int64)
    for r in range(n_parts):
        owner[order[bounds[r]:bounds[r + 1]]] = r
    return owner


def shard_masks(levels_coords, rank: int, n_ranks: int):
    """Per level, the boolean mask of the blocks that rank owns."""
    return [morton_partition(c, n_ranks) == rank for c in levels_coords]
