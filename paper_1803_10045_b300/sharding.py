"""Plane sharding of a stacked-2D study across ranks (host logic only).

The projector rays, the OSL update and the in-plane 3x3 Huber cliques never
couple two planes, so an ICM run on a contiguous plane range is exactly the
full run restricted to those planes: ranks need no data exchange, only their
own plane range.  The optional 26-neighbour (3x3x3) Huber prior couples
adjacent planes; with it, halo_exchange supplies the one-plane halo of the
kinetic maps once per MAP-LM step.
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


def halo_exchange(local, rank: int, world: int, halo: int = 1, group=None):
    """Attach the neighbouring ranks' boundary planes to a plane-sharded array.

    local: a tensor [..., Z_local, Y, X] (plane axis -3) holding this rank's
    contiguous plane range (plane_shard order).  Returns (padded, lo, hi):
    padded = [..., lo + Z_local + hi, Y, X] with `lo` planes received from
    rank - 1 below and `hi` planes from rank + 1 above (0 at the ends of the
    volume).  This is the one exchange the path needs, and only with the
    26-neighbour (3x3x3) Huber prior: once per MAP-LM step for the 4 maps, so
    that every rank sees its neighbours' start-of-step values (the synchronous
    update); the in-plane prior needs none.  Point-to-point send/recv through
    torch.distributed (gloo on the CPU, NCCL on GPUs).
    """
    import torch
    import torch.distributed as dist
    if local.shape[-3] < halo:
        raise ValueError("each rank needs at least `halo` planes")
    reqs = []
    lo_buf = hi_buf = None
    if rank > 0:
        lo_buf = torch.empty_like(local[..., :halo, :, :].contiguous())
        reqs.append(dist.irecv(lo_buf, rank - 1, group=group))
        reqs.append(dist.isend(local[..., :halo, :, :].contiguous(), rank - 1, group=group))
    if rank < world - 1:
        hi_buf = torch.empty_like(local[..., -halo:, :, :].contiguous())
        reqs.append(dist.irecv(hi_buf, rank + 1, group=group))
        reqs.append(dist.isend(local[..., -halo:, :, :].contiguous(), rank + 1, group=group))
    for r in reqs:
        r.wait()
    parts = [p for p in (lo_buf, local, hi_buf) if p is not None]
    return torch.cat(parts, dim=-3), (halo if lo_buf is not None else 0), \
        (halo if hi_buf is not None else 0)
