"""Differentiable forward model y = P F(theta) (config PR4 pattern) on the GPU.

The backward pass is the library's exact back-projection composed with the
analytic kinetic Jacobian transposed (kcs_tac_vjp).  Checked against (1) the
Jacobian that kcs_tac_eval returns, (2) the FP64 oracle's gradient J^T P^T w,
(3) central finite differences (h = 1e-3) on 256 random voxels, and (4) 50
gradient-MAP steps that must lower the Poisson + Huber objective.
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import kinetics as OK
from oracle import projector as OP
from cases import rel_l2

pytestmark = pytest.mark.gpu
SCHED = "m16"      # 4x15 s, 4x60 s, 4x180 s, 4x300 s


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _theta(shape, seed):
    rng = np.random.default_rng(seed)
    base = np.array(S.CLASS_XI["gm"])[:, None, None, None]
    return np.clip(base * rng.uniform(0.5, 1.5, (4,) + shape), 0, [[[[2]]], [[[2]]], [[[1]]], [[[1]]]])


def test_vjp_matches_jacobian(cuda_ok):
    import paper_1803_10045_b300 as K
    ts, te = S.schedule(S.SCHEDULES[SCHED])
    kin = K.Kinetics(ts, te, S.FENG)
    p = _t(_theta((3, 17, 19), 0))
    gF = torch.randn((3, 17, 19, 16), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    F, J = K.tac_eval(kin, p, jacobian=True)
    ref = torch.einsum("zyxmq,zyxm->qzyx", J.double(), gF.double())
    got = K.tac_vjp(kin, p, gF).double()
    assert rel_l2(got.cpu().numpy(), ref.cpu().numpy()) < 1e-6


def test_gradient_matches_oracle(cuda_ok):
    import paper_1803_10045_b300 as K
    nx, nz, B, A = 20, 2, 29, 18
    ts, te = S.schedule(S.SCHEDULES[SCHED])
    kg = K.Geometry(nx, nx, nz, 2.0, B, A, 2.0, 3)
    og = OP.Geometry(nx, nx, 2.0, B, A, 2.0, 3)
    kin = K.Kinetics(ts, te, S.FENG)
    th = np.asarray(_theta((nz, nx, nx), 2), np.float32).astype(np.float64)
    w = np.random.default_rng(3).uniform(-1, 1, (nz, A, B, 16))
    tht = _t(th).requires_grad_(True)
    y = K.forward_model(tht, kg, kin)
    (y * _t(w)).sum().backward()
    # oracle: dL/dtheta = J^T (P^T w)
    gF = og.back(w)                                         # [Z][Y][X][M]
    _, J = OK.model(th.reshape(4, -1).T, ts, te, S.FENG)    # [V][M][4]
    ref = np.einsum("vmq,vm->qv", J, gF.reshape(-1, 16)).reshape(th.shape)
    assert rel_l2(tht.grad.double().cpu().numpy(), ref) < 1e-4
    # and the forward value itself
    Fo = OK.model_maps(th, ts, te, S.FENG)
    assert rel_l2(y.detach().double().cpu().numpy(), og.forward(Fo)) < 1e-5


# sizes: batch, image side, planes, bins, angles; "pr4" is the full config PR4
# (theta [8][4][64][128][128], 128 bins x 96 angles, 16 frames)
SIZES = {"small": (2, 32, 4, 45, 24), "pr4": (8, 128, 64, 128, 96)}


@pytest.mark.parametrize("size", ["small", "pr4"])
def test_central_differences_on_256_voxels(cuda_ok, size):
    import paper_1803_10045_b300 as K
    nb, nx, nz, B, A = SIZES[size]
    ts, te = S.schedule(S.SCHEDULES[SCHED])
    kg = K.Geometry(nx, nx, nb * nz, 2.0, B, A, 2.0, 1)
    kin = K.Kinetics(ts, te, S.FENG)
    th = _t(np.stack([_theta((nz, nx, nx), 10 + b) for b in range(nb)]))   # [B][4][Z][Y][X]
    w = torch.rand((nb, nz, A, B, 16), device="cuda", generator=torch.Generator("cuda").manual_seed(4))

    def loss(t):
        return (K.forward_model(t, kg, kin).double() * w.double()).sum()

    t = th.clone().requires_grad_(True)
    loss(t).backward()
    g = t.grad.double().cpu().numpy()
    rng = np.random.default_rng(5)
    h = 1e-3
    errs = []
    with torch.no_grad():
        for _ in range(256):
            b, z, j, i = (int(rng.integers(nb)), int(rng.integers(nz)), int(rng.integers(nx)),
                          int(rng.integers(nx)))
            q = int(rng.integers(4))
            tp, tm = th.clone(), th.clone()
            tp[b, q, z, j, i] += h
            tm[b, q, z, j, i] -= h
            fd = (loss(tp) - loss(tm)).item() / (2 * h)
            ref = g[b, q, z, j, i]
            errs.append(abs(fd - ref) / max(abs(ref), 1e-2 * np.abs(g[:, q]).max()))
    assert np.median(errs) < 1e-3 and np.max(errs) < 3e-2, (np.median(errs), np.max(errs))


@pytest.mark.parametrize("size", ["small", "pr4"])
def test_gradient_map_lowers_objective(cuda_ok, size):
    import paper_1803_10045_b300 as K
    nb, nx, nz, B, A = SIZES[size]
    ts, te = S.schedule(S.SCHEDULES[SCHED])
    kg = K.Geometry(nx, nx, nb * nz, 2.0, B, A, 2.0, 1)
    kin = K.Kinetics(ts, te, S.FENG)
    truth = _t(np.stack([_theta((nz, nx, nx), 20 + b) for b in range(nb)]))
    dt = _t(te - ts)
    with torch.no_grad():
        ybar = K.forward_model(truth, kg, kin) * dt * 20.0
        counts = torch.poisson(ybar + 0.5, generator=torch.Generator("cuda").manual_seed(6))
    lo = torch.zeros(4, device="cuda")[None, :, None, None, None]
    hi = torch.tensor([2.0, 2.0, 1.0, 1.0], device="cuda")[None, :, None, None, None]
    th = (truth * 0 + torch.tensor(S.XI0, device="cuda")[None, :, None, None, None]).requires_grad_(True)
    opt = torch.optim.Adam([th], lr=5e-3)
    delta, beta = 0.01, 0.1

    def huber(t):
        e = 0.0
        for dy, dx in ((0, 1), (1, 0), (1, 1), (1, -1)):
            a = t[..., max(dy, 0):t.shape[-2] + min(dy, 0), max(dx, 0):t.shape[-1] + min(dx, 0)]
            b = t[..., max(-dy, 0):t.shape[-2] + min(-dy, 0), max(-dx, 0):t.shape[-1] + min(-dx, 0)]
            d = (a - b).abs()
            e = e + torch.where(d <= delta, 0.5 * d * d, delta * d - 0.5 * delta * delta).sum()
        return e

    def objective(t):
        yb = K.forward_model(t, kg, kin) * dt * 20.0 + 0.5
        return (yb - counts * torch.log(yb)).sum() + beta * huber(t)

    first = None
    for _ in range(50):
        opt.zero_grad()
        f = objective(th)
        if first is None:
            first = f.item()
        f.backward()
        opt.step()
        with torch.no_grad():
            th.copy_(torch.maximum(torch.minimum(th, hi), lo))
    last = objective(th).item()
    print(f"gradient-MAP: objective {first:.6e} -> {last:.6e}")
    assert last < first - 1e-3 * abs(first)
