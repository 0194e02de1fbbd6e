"""Replica (data-parallel) runs: shard plan and the final entity-map union.

Records are independent, windows never cross records and a pseudonym is a
function of the key and the entity bytes alone (AnonShield §2 stage (4)), so
replicas need no communication while they process. The only exchange is the
union of their entity maps at the end: each rank exports its map, rank 0
gathers them over torch.distributed (gloo or NCCL; objects, not tensors) and
merges them with as_map_merge, shifting each replica's record indices by the
global index of its first record.
"""
from __future__ import annotations

import numpy as np

from . import api


def shard_ranges(record_bytes: np.ndarray, world: int) -> list[tuple[int, int]]:
    """Contiguous record ranges [start, end), one per rank, balanced by bytes.

    Bytes stand in for tokens (known only after tokenizing). Boundary r is the
    first record whose byte prefix sum reaches r/world of the total.
    """
    n = len(record_bytes)
    if world <= 1:
        return [(0, n)]
    csum = np.concatenate([[0], np.cumsum(np.asarray(record_bytes, dtype=np.int64))])
    total = int(csum[-1])
    cuts = [0]
    for r in range(1, world):
        cuts.append(max(cuts[-1], int(np.searchsorted(csum, total * r / world, side="left"))))
    cuts.append(n)
    cuts = [min(c, n) for c in cuts]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def _pack(entries: list[api.Entity]) -> list[tuple]:
    return [(e.type, e.original, e.full_hash, e.slug, e.first_seen, e.last_seen, e.count) for e in entries]


def gather_merge(entries: list[api.Entity], record_offset: int, group=None) -> list[api.Entity] | None:
    """Union of every rank's map on rank 0 (None on the other ranks)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mine = (int(record_offset), _pack(entries))
    got = [None] * world if rank == 0 else None
    dist.gather_object(mine, got, dst=0, group=group)
    if rank != 0:
        return None
    shards = [[api.Entity(*t) for t in g[1]] for g in got]
    return api.map_merge(shards, [g[0] for g in got])
