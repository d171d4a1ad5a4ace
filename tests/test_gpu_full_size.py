"""Full-size parity (GPU): the fused OSL update and the MAP-LM step on the PR2
workload's geometry (344 x 344 x 127 voxels, 344 bins x 252 angles, 21
subsets, 24 frames), in the launch configuration the benchmark times, checked
against the FP64 oracle on outputs it can compute independently: whole planes
of the OSL update (planes do not interact) and single voxels of the LM step
(a voxel's step depends only on its own TAC and its 3 x 3 in-plane
neighbourhood).  Inputs are seeded and synthetic; the oracle receives the
same float32 values.
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from cases import lm_step_parity, rel_l2, ulp
from oracle import kinetics as OK
from oracle import lm as OL
from oracle import osl as OO
from oracle import projector as OP

pytestmark = pytest.mark.gpu


def _f32(v):
    return float(np.float32(v))


# beta = 0.05 makes the prior up to ~8 % of the data term kappa dt sens in the
# 15 s frames.  A prior comparable to the data term can bring the OSL
# denominator within a small factor of its 1e-3 clamp (measured with beta = 0.5:
# updates x_new / x up to 2e4), where float32 rounding of the denominator is
# amplified by the same factor (rel-L2 1.3e-4 against the oracle there,
# 2.6e-6 here).
@pytest.mark.parametrize("beta", [0.0, 0.05])
def test_full_size_osl_update_planes(cuda_ok, beta):
    import paper_1803_10045_b300 as K
    W = S.WORKLOADS["pr2"]
    M, k = W.n_frames, 11
    kg = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    og = OP.Geometry(W.nx, W.ny, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    ts, te = W.frames()
    dt = np.asarray(te - ts, np.float32)
    kappa = _f32(2e-3)
    gen = torch.Generator(device="cuda").manual_seed(11)
    shape = (W.nz, W.ny, W.nx, M)
    x = 0.5 + 2.0 * torch.rand(shape, device="cuda", generator=gen)
    F = x * (0.8 + 0.4 * torch.rand(shape, device="cuda", generator=gen))
    counts_i = torch.randint(0, 12, (W.nz, W.n_angles, W.n_bins, M), device="cuda",
                             generator=gen, dtype=torch.int32)
    counts = counts_i.to(torch.uint16)                     # the benchmark's counts type
    r = (0.05 * dt).astype(np.float32)                     # randoms per frame
    zs = [0, 63, 126]
    x0 = x[zs].double().cpu().numpy()
    F0 = F[zs].double().cpu().numpy()
    ang = og.subsets[k]
    c0 = counts_i[zs][:, torch.as_tensor(ang, device="cuda")].double().cpu().numpy()
    K.osl_update(kg, k, x, torch.tensor(dt, device="cuda"), kappa, counts,
                 torch.tensor(r, device="cuda"), None, F, beta, 1.0)
    got = x[zs].double().cpu().numpy()
    ref = OO.osl_update(og, x0, k, c0, kappa, dt.astype(np.float64), None,
                        r.astype(np.float64), F0, beta, 1.0)
    for n, z in enumerate(zs):
        e = rel_l2(got[n], ref[n])
        print(f"beta {beta} plane {z}: rel-L2 {e:.2e}")
        assert e < 1e-4


@pytest.mark.parametrize("kind", ["bf16", "f16"])
def test_full_size_stored_osl_update_planes(cuda_ok, kind):
    """The precision form at full size: the fused OSL update of an image stored
    as bfloat16 / float16 with a per-frame scale (uint16 counts, the prior on)
    equals, on three whole planes, the oracle's update with the same stores
    rounded to the same grid, within one unit in the last place of the
    storage type."""
    import paper_1803_10045_b300 as K
    W = S.WORKLOADS["pr2"]
    M, k, beta = W.n_frames, 11, 0.05
    kg = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    og = OP.Geometry(W.nx, W.ny, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    ts, te = W.frames()
    dt = np.asarray(te - ts, np.float32)
    kappa = _f32(2e-3)
    gen = torch.Generator(device="cuda").manual_seed(13)
    shape = (W.nz, W.ny, W.nx, M)
    x = 0.5 + 2.0 * torch.rand(shape, device="cuda", generator=gen)
    F = x * (0.8 + 0.4 * torch.rand(shape, device="cuda", generator=gen))
    counts_i = torch.randint(0, 12, (W.nz, W.n_angles, W.n_bins, M), device="cuda",
                             generator=gen, dtype=torch.int32)
    counts = counts_i.to(torch.uint16)
    r = (0.05 * dt).astype(np.float32)
    scale = x.reshape(-1, M).amax(0)                        # per-frame level, float32
    xs = (x / scale).to({"bf16": torch.bfloat16, "f16": torch.float16}[kind])
    del x
    zs = [0, 63, 126]
    ang = torch.as_tensor(og.subsets[k], device="cuda")
    xs0 = xs[zs].double().cpu().numpy()
    F0 = F[zs].double().cpu().numpy()
    c0 = counts_i[zs][:, ang].double().cpu().numpy()
    del counts_i
    sc = scale.double().cpu().numpy()
    K.osl_update(kg, k, xs, torch.tensor(dt, device="cuda"), kappa, counts,
                 torch.tensor(r, device="cuda"), None, F, beta, 1.0, x_scale=scale)
    got = xs[zs].double().cpu().numpy()
    ref = OO.osl_update_stored(og, xs0, k, c0, kappa, dt.astype(np.float64), sc, kind,
                               randoms_k=r.astype(np.float64), F=F0, beta=beta)
    nulp = np.abs(got - ref) / ulp(ref, kind)
    print(f"{kind}: max {nulp.max():.2f} ulp, {np.mean(nulp > 0):.3%} of values differ")
    assert nulp.max() <= 1.0 + 1e-9
    assert np.mean(nulp > 0) < 0.02


def test_full_size_lm_step_sampled_voxels(cuda_ok):
    import paper_1803_10045_b300 as K
    W = S.WORKLOADS["pr2"]
    ts, te = W.frames()
    M = W.n_frames
    beta, delta = 0.1, 0.01
    kin = K.Kinetics(ts, te, S.FENG)
    # start maps: the brain-like phantom; TACs: per-voxel mixtures of the grey-
    # and white-matter model curves (oracle, float64 -> float32)
    gen = torch.Generator(device="cuda").manual_seed(12)
    maps0 = torch.tensor(S.phantom_pr2(W.nx, W.nz, seed=1), device="cuda")
    # start points spread over a factor 3 around the phantom, lambda over 1e-6..10,
    # so that the step both accepts and rejects
    maps0 *= 0.5 + torch.rand(maps0.shape, device="cuda", generator=gen)
    curves = OK.model(np.array([S.CLASS_XI["gm"], S.CLASS_XI["wm"]], float), ts, te, S.FENG,
                      jacobian=False)
    c = torch.tensor(curves, dtype=torch.float32, device="cuda")
    vshape = (W.nz, W.ny, W.nx)
    a = 0.2 + torch.rand(vshape + (2,), device="cuda", generator=gen)
    x = (a[..., 0:1] * c[0] + a[..., 1:2] * c[1]).contiguous()
    lam0 = 10.0 ** (-6.0 + 7.0 * torch.rand(vshape, device="cuda", generator=gen))
    p, lam = maps0.clone(), lam0.clone()
    K.map_lm_fit(kin, x, p, 1, beta, delta, lam=lam)
    torch.cuda.synchronize()

    # interior voxels (full 3 x 3 neighbourhood), 70 % inside the head
    rng = np.random.default_rng(12)
    n = 800
    head = (maps0[0] > 0).nonzero().cpu().numpy()
    head = head[(head[:, 1] > 0) & (head[:, 1] < W.ny - 1) & (head[:, 2] > 0) & (head[:, 2] < W.nx - 1)]
    pick = head[rng.choice(len(head), int(0.7 * n), replace=False)]
    anyv = np.stack([rng.integers(0, W.nz, n), rng.integers(1, W.ny - 1, n),
                     rng.integers(1, W.nx - 1, n)], 1)[: n - len(pick)]
    zji = torch.tensor(np.concatenate([pick, anyv]), device="cuda")
    d = torch.arange(-1, 2, device="cuda")
    zz = zji[:, 0, None, None]
    jj = zji[:, 1, None, None] + d[None, :, None]
    ii = zji[:, 2, None, None] + d[None, None, :]
    win_maps = maps0[:, zz, jj, ii].double().cpu().numpy()          # [4][n][3][3]
    win_x = x[zz, jj, ii].double().cpu().numpy()                     # [n][3][3][M]
    win_lam = lam0[zz, jj, ii].double().cpu().numpy()
    got = p[:, zji[:, 0], zji[:, 1], zji[:, 2]].double().cpu().numpy().T   # [n][4]
    lam_g = lam[zji[:, 0], zji[:, 1], zji[:, 2]].double().cpu().numpy()
    # the oracle's step of each window (3 x 3 neighbourhoods as separate planes);
    # the centre voxel of window k is voxel 9 k + 4 of the flattened result
    sp = OL.float32_spread(win_x, win_maps, win_lam, ts, te, S.FENG, beta, delta)
    ctr = np.arange(n) * 9 + 4
    keys = ("acc", "trial", "xi", "flip", "margin", "dev_trial", "dev_margin", "model_margin",
            "huber_margin")
    spc = {k: sp[k][ctr] for k in keys}
    # lambda spans 1e-6 .. 10 here, so more steps are float32-sensitive than on
    # PR1 (the share is fixed by the oracle: 73 % strict on these inputs)
    lm_step_parity(got.T, lam_g, win_lam[:, 1, 1], spc, 0.6, "PR2 sampled voxels")


def test_full_size_plane_shards_equal_full_volume(cuda_ok):
    """Plane sharding of the product path at full size: the CUDA ICM run on
    each rank's contiguous plane range (plane_shard, 4 ranks, emulated one
    after another on this GPU) equals the full 127-plane run restricted to
    those planes bit for bit, image, maps and model TACs.  No cross-plane
    term exists in the projector, the OSL update, the in-plane Huber prior or
    the LM step, so a multi-GPU run needs no data-path exchange.  The start
    image is the full volume's (its per-frame level is a sum over all planes)."""
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300.sharding import plane_shard
    W = S.WORKLOADS["pr2"]
    ts, te = W.frames()
    M = W.n_frames
    g = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    kin = K.Kinetics(ts, te, S.FENG)
    dt = torch.tensor(te - ts, dtype=torch.float32, device="cuda")
    xi = torch.tensor(S.phantom_pr2(W.nx, W.nz, seed=3), device="cuda")
    ybar = K.forward_project(g, K.tac_eval(kin, xi)).mul_(dt)
    kappa = _f32(W.total_prompts * (1 - W.randoms_frac) / ybar.double().sum().item())
    r = (W.total_prompts * W.randoms_frac) * dt / (dt.sum() * W.nz * W.n_angles * W.n_bins)
    counts = torch.poisson(ybar.mul_(kappa).add_(r),
                           generator=torch.Generator(device="cuda").manual_seed(3))
    del ybar, xi
    counts = counts.to(torch.uint16)                       # the benchmark's counts type
    x0 = K.init_image(g, dt, kappa, counts, r)
    p0 = torch.empty((4, W.nz, W.ny, W.nx), device="cuda")
    p0[:] = torch.tensor(S.XI0, device="cuda")[:, None, None, None]
    kw = dict(randoms=r, n_lm=10, beta_kp=0.1, beta_h=0.1, delta=0.01)

    def run(geom, c, x, p):
        F = torch.zeros(x.shape, device="cuda")
        K.Study(geom, kin, dt, kappa, c, x, p, F=F, **kw).iterate(2)
        return F
    x, p = x0.clone(), p0.clone()
    F = run(g, counts, x, p)
    world = 4
    for rank in range(world):
        z0, z1 = plane_shard(W.nz, rank, world)
        gs = K.Geometry(W.nx, W.ny, z1 - z0, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm,
                        W.n_subsets)
        xs, ps = x0[z0:z1].clone(), p0[:, z0:z1].contiguous()
        Fs = run(gs, counts[z0:z1].contiguous(), xs, ps)
        torch.cuda.synchronize()
        assert torch.equal(xs, x[z0:z1]), f"rank {rank} image"
        assert torch.equal(ps, p[:, z0:z1]), f"rank {rank} maps"
        assert torch.equal(Fs, F[z0:z1]), f"rank {rank} model TACs"
