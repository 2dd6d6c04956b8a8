"""Partition of the path over ranks (one GPU per rank).

Subbands are independent after channelisation and (target, subband) pairs
are independent problems, so ranks need no exchange: rank r takes a
contiguous block of subbands (or of whole batches).  Host logic only.
"""
from __future__ import annotations


def shard_range(n: int, world: int, rank: int) -> range:
    """Balanced contiguous block of range(n) for `rank` of `world`:
    the first n % world ranks get one extra item."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def shard_subbands(L: int, world: int, rank: int) -> list:
    """Subband indices handled by `rank`."""
    return list(shard_range(L, world, rank))
