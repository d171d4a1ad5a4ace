"""Plane sharding of a stacked-2D study across ranks (host logic only).

The projector rays, the OSL update and the in-plane 3x3 Huber cliques never
couple two planes, so an ICM run on a contiguous plane range is exactly the
full run restricted to those planes: ranks need no data exchange, only their
own plane range.
"""
from __future__ import annotations


def plane_shard(nz: int, rank: int, world: int):
    """Contiguous plane range [z0, z1) of `rank` among `world` ranks; the first
    nz % world ranks take one extra plane."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)
