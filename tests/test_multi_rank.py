"""Plane sharding across ranks (CPU, gloo, world size 2).

Each rank runs the ICM on its own contiguous plane range and the gathered
result equals the unsharded run: the path has no cross-plane coupling, so a
multi-GPU run needs no data-path collective.  (Equality is to rounding: the
uniform start image's per-frame level is a sum over the planes a rank sees,
and the first multiplicative OSL update removes that level exactly only in
exact arithmetic.)  The per-rank work
is the float64 oracle here (no GPU in this test); the GPU kernels index planes
the same way (every launch covers whole planes).
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import kcs_synth as S
from paper_1803_10045_b300.sharding import plane_shard


def _problem():
    from oracle import kinetics as OK
    from oracle import projector as OP
    nx, nz, B, A, Sb = 16, 5, 24, 20, 2
    g = OP.Geometry(nx, nx, 2.0, B, A, 2.0, Sb)
    ts, te = S.schedule([(2, 60), (2, 300)])
    rng = np.random.default_rng(0)
    xi = np.clip(S.CLASS_XI["gm"] * rng.uniform(0.5, 1.5, (nz, nx, nx, 4)), 0, None)
    xi = np.moveaxis(xi, -1, 0)
    F = OK.model_maps(xi, ts, te, S.FENG)
    counts = S.poisson(g.forward(F) * (te - ts) * 50.0, 1)
    return g, ts, te, counts


def _run(counts, g, ts, te):
    from oracle import icm as OI
    x, xi, _, _ = OI.icm(g, counts, 50.0, ts, te, S.FENG, 2, 2, 0.1, 0.1, 0.01)
    return x, xi


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, ts, te, counts = _problem()
    z0, z1 = plane_shard(counts.shape[0], rank, world)
    x, xi = _run(counts[z0:z1], g, ts, te)
    parts = [None] * world
    dist.all_gather_object(parts, (z0, z1, x, xi))
    if rank == 0:
        np.save(out, np.array([p for p in parts], dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_plane_shard_covers_planes():
    for nz in (1, 5, 127):
        for world in (1, 2, 3, 8):
            r = [plane_shard(nz, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == nz
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
            assert max(b - a for a, b in r) - min(b - a for a, b in r) <= 1
    with pytest.raises(ValueError):
        plane_shard(5, 2, 2)


def test_sharded_icm_equals_unsharded(tmp_path):
    out = str(tmp_path / "parts.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    parts = np.load(out, allow_pickle=True)
    g, ts, te, counts = _problem()
    x, xi = _run(counts, g, ts, te)
    for z0, z1, xs, xis in parts:
        np.testing.assert_allclose(xs, x[z0:z1], rtol=1e-11, atol=0)
        np.testing.assert_allclose(xis, xi[:, z0:z1], rtol=1e-9, atol=1e-14)


def _lm_problem():
    from oracle import kinetics as OK
    nx, nz = 12, 5
    ts, te = S.schedule([(2, 60), (2, 300)])
    rng = np.random.default_rng(3)
    xi = np.moveaxis(np.clip(S.CLASS_XI["gm"] * rng.uniform(0.5, 1.5, (nz, nx, nx, 4)), 0, None),
                     -1, 0)
    x = OK.model_maps(xi, ts, te, S.FENG) * (1 + 0.05 * rng.standard_normal((nz, nx, nx, 4)))
    start = np.clip(xi * rng.uniform(0.8, 1.2, xi.shape), 0, None)
    return x, start, ts, te


def _lm_worker(rank, world, port, out):
    import torch
    from oracle import lm as OL
    from paper_1803_10045_b300.sharding import halo_exchange
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, start, ts, te = _lm_problem()
    z0, z1 = plane_shard(x.shape[0], rank, world)
    maps = start[:, z0:z1].copy()
    lam = np.full(maps.shape[1:], OL.LAMBDA0)
    # the TAC halo is exchanged once (it does not change during the fit)
    xp, xl, xh = halo_exchange(torch.from_numpy(np.moveaxis(x[z0:z1], -1, 0).copy()), rank, world)
    xp = np.moveaxis(xp.numpy(), 0, -1)
    for _ in range(3):
        mp_, lo, hi = halo_exchange(torch.from_numpy(maps), rank, world)
        lam_p = np.pad(lam, ((lo, hi), (0, 0), (0, 0)), constant_values=OL.LAMBDA0)
        new, lam_new, _, _ = OL.lm_step(xp, mp_.numpy(), lam_p, ts, te, S.FENG, 0.5, 0.01,
                                        nbhd="3d")
        sl = slice(lo, lo + (z1 - z0))
        maps, lam = new[:, sl].copy(), lam_new[sl].copy()
    parts = [None] * world
    dist.all_gather_object(parts, (z0, z1, maps))
    if rank == 0:
        np.save(out, np.array(parts, dtype=object), allow_pickle=True)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_3d_prior_lm_with_halo_equals_unsharded(tmp_path):
    """With the 26-neighbour prior the planes couple; a one-plane halo of the 4
    maps exchanged per LM step makes the sharded fit equal the unsharded one."""
    from oracle import lm as OL
    out = str(tmp_path / "lm_parts.npy")
    mp.start_processes(_lm_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    parts = np.load(out, allow_pickle=True)
    x, start, ts, te = _lm_problem()
    ref, _ = OL.lm_fit(x, start, 3, ts, te, S.FENG, 0.5, 0.01, nbhd="3d")
    got = np.concatenate([p[2] for p in sorted(parts, key=lambda p: p[0])], axis=1)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15)
    # and without the halo the result would differ (the exchange matters)
    alone = np.concatenate([OL.lm_fit(x[a:b], start[:, a:b], 3, ts, te, S.FENG, 0.5, 0.01,
                                      nbhd="3d")[0] for a, b in ((0, 3), (3, 5))], axis=1)
    assert not np.allclose(alone, ref, rtol=1e-9)
