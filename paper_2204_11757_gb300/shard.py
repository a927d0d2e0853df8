"""Sharding a batch of independent graphs across ranks (one process per GPU).

Graphs of a batch share nothing, so the batched path splits them into contiguous ranges of
roughly equal edge count, one range per rank, with no exchange during coarsening.  The only
collective is a final all-gather of the per-graph super-node counts (B integers), which gives
every rank the global super-node offsets.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def shard_ranges(edge_counts: np.ndarray, world_size: int) -> List[Tuple[int, int]]:
    """Contiguous graph ranges [g0, g1) per rank, split at cumulative-edge-count quantiles.

    Every graph goes to exactly one rank; ranks may be empty only when B < world_size.
    """
    edge_counts = np.asarray(edge_counts, dtype=np.int64)
    B = int(edge_counts.shape[0])
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    cum = np.concatenate([[0], np.cumsum(edge_counts)])
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world_size):
        target = total * r / world_size
        g = int(np.searchsorted(cum, target, side="left"))
        g = min(max(g, cuts[-1]), B)
        cuts.append(g)
    cuts.append(B)
    return [(cuts[r], cuts[r + 1]) for r in range(world_size)]


def batch_edge_counts(batch) -> np.ndarray:
    """Undirected edges of every graph of a block-diagonal batch."""
    g = batch.graph
    stored = g.rowptr[batch.graph_ptr[1:]] - g.rowptr[batch.graph_ptr[:-1]]
    return (stored // 2).astype(np.int64)


def local_batch(batch, rank: int, world_size: int):
    """This rank's sub-batch and its global graph range."""
    from .inputs import subsample_batch
    g0, g1 = shard_ranges(batch_edge_counts(batch), world_size)[rank]
    return subsample_batch(batch, np.arange(g0, g1)), (g0, g1)


def global_offsets(local_counts: np.ndarray, ranges, world_size: int, all_gather=None):
    """Global super-node offsets from every rank's per-graph counts.

    `all_gather(tensor_list, tensor)` is torch.distributed.all_gather (or None for one rank).
    Returns int64[B+1] offsets, identical on every rank.
    """
    import torch
    B = ranges[-1][1]
    sizes = [r[1] - r[0] for r in ranges]
    width = max(sizes) if sizes else 0
    mine = torch.full((width,), -1, dtype=torch.int64)
    mine[:len(local_counts)] = torch.as_tensor(np.asarray(local_counts, dtype=np.int64))
    if all_gather is None or world_size == 1:
        parts = [mine]
    else:
        parts = [torch.empty_like(mine) for _ in range(world_size)]
        all_gather(parts, mine)
    counts = np.zeros(B, dtype=np.int64)
    for (g0, g1), p in zip(ranges, parts):
        counts[g0:g1] = p[:g1 - g0].numpy()
    off = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off
