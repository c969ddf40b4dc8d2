"""Root-range sharding of one query over several GPUs.

The embeddings of Q in G partition by the data vertex M[phi[0]] that the
first query vertex of the matching order maps to, so disjoint root ranges
give disjoint embedding sets whose counts and hashes add up (the hash is a
sum mod 2^64). Each rank holds a replica of G and counts its own range; no
data moves between ranks until the final 16-byte sums.
"""
from __future__ import annotations

MASK64 = (1 << 64) - 1


def root_range(n: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous vertex-id range [lo, hi) of rank `rank` out of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return rank * n // world, (rank + 1) * n // world


def combine(parts):
    """Sums per-shard (count, hash) pairs: the hash wraps mod 2^64."""
    count, h = 0, 0
    for c, x in parts:
        count += int(c)
        h = (h + int(x)) & MASK64
    return count, h
