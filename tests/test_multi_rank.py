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
