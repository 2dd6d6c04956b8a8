"""Partition of the path over ranks (one GPU per rank).

Subbands are independent after channelisation and (target, subband) pairs
are independent problems, so ranks need no exchange: rank r takes a
contiguous block of subbands (or of whole batches).  A library plan covers
an aligned power-of-two block of subbands (bs_config.s_begin, s_count), so a
rank's block is split into such blocks, one plan each.  Host logic only.
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


def aligned_blocks(begin: int, end: int) -> list:
    """[begin, end) as maximal aligned power-of-two blocks (s_begin, s_count):
    every s_count is a power of two and s_begin a multiple of it, the blocks
    are disjoint, in order, and cover the range exactly."""
    if begin < 0 or end < begin:
        raise ValueError("need 0 <= begin <= end")
    out, s = [], begin
    while s < end:
        size = s & -s if s else 1 << (end - 1).bit_length()
        while size > end - s:
            size >>= 1
        out.append((s, size))
        s += size
    return out


def shard_plan_blocks(L: int, world: int, rank: int) -> list:
    """(s_begin, s_count) of the plans that run `rank`'s subbands: its
    balanced contiguous block of range(L), split into aligned power-of-two
    blocks (one block when world is a power of two dividing L)."""
    r = shard_range(L, world, rank)
    return aligned_blocks(r.start, r.stop)
