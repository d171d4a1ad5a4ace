"""CUDA Huber prior and MAP-LM step vs the FP64 oracle (GPU).

Teacher-forced parity: both sides take one synchronous LM step from the same
maps, lambda and TACs.  Where both accept, the new maps agree within 1e-3 of
max(|xi_ref|, floor_p) per voxel (floor_p = 1e-2 x the parameter's class mean,
because k2 and k3 are unidentifiable where the tissue term vanishes); where
both reject, the maps are unchanged.  Accept/reject decisions taken in
float32 vs float64 may differ where the objective barely changes; their count
is bounded, not required to be zero.
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import kinetics as OK
from oracle import lm as OL
from cases import pr1_problem

pytestmark = pytest.mark.gpu
FLOOR = 1e-2 * np.array([0.06, 0.10, 0.04, 0.03])


def _t(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


@pytest.mark.parametrize("delta", [0.01, 1e30])
def test_huber_grad_matches_oracle(cuda_ok, delta):
    import paper_1803_10045_b300 as K
    rng = np.random.default_rng(3)
    maps = rng.uniform(0, 0.1, (4, 3, 17, 23))
    got = K.huber_grad(_t(maps), delta).double().cpu().numpy()
    ref = OL.huber_grad(_f32(maps), delta)
    np.testing.assert_allclose(got, ref, atol=2e-6)


def _lm_case(seed=0):
    P = pr1_problem()
    rng = np.random.default_rng(seed)
    # image TACs: the noisy truth; start maps: jittered truth (class values)
    x = P["Ftrue"] * (1 + 0.05 * rng.standard_normal(P["Ftrue"].shape))
    maps = np.clip(P["xi"] * rng.uniform(0.7, 1.3, P["xi"].shape), 0, None)
    maps[:, P["xi"][0] == 0] = np.array(S.XI0)[:, None]
    lam = 10.0 ** rng.uniform(-4, 0, maps.shape[1:])
    return P, _f32(x), _f32(maps), _f32(lam)


@pytest.mark.parametrize("beta", [0.0, 0.1, 50.0])
def test_single_step_teacher_forced(cuda_ok, beta):
    import paper_1803_10045_b300 as K
    P, x, maps, lam = _lm_case()
    kin = K.Kinetics(P["ts"], P["te"], S.FENG)
    pg, lg = _t(maps), _t(lam)
    K.map_lm_fit(kin, _t(x), pg, 1, beta, 0.01, lam=lg)
    got = pg.double().cpu().numpy()
    lam_g = lg.double().cpu().numpy()
    ref, lam_r, acc_r, _ = OL.lm_step(x, maps, lam, P["ts"], P["te"], S.FENG, beta, 0.01)
    acc_g = np.isclose(lam_g, np.maximum(lam / 10, 1e-7), rtol=1e-5)
    agree = acc_g == acc_r
    print(f"beta={beta}: accept agreement {agree.mean():.4f}, accepted {acc_r.mean():.3f}")
    assert agree.mean() > 0.99, (agree.mean(), (~agree).sum())
    tol = 1e-3 * np.maximum(np.abs(ref), FLOOR[:, None, None, None])
    within = np.all(np.abs(got - ref) <= tol, axis=0)[agree]
    # a voxel on a flat valley (k2, k3 unidentifiable where the tissue term is
    # small) turns the float32 model's rounding into a large step difference;
    # bound the share of such voxels instead of requiring none
    print(f"beta={beta}: maps within 1e-3 on {within.mean():.5f} of the voxels")
    assert within.mean() > 0.999
    rej = ~acc_g & ~acc_r
    np.testing.assert_array_equal(got[:, rej], maps[:, rej])


def test_noise_free_recovery(cuda_ok):
    import paper_1803_10045_b300 as K
    ts, te = S.schedule(S.SCHEDULES["pr2"])
    xi = np.clip(S.jittered_params(256, seed=8, rel=0.3), 0, [2, 2, 1, 1])
    F = OK.model(_f32(xi), ts, te, S.FENG, jacobian=False)
    kin = K.Kinetics(ts, te, S.FENG)
    x = _t(F.reshape(1, 16, 16, -1))
    p = _t(np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 16, 16)))
    K.map_lm_fit(kin, x, p, 60, 0.0, 0.01)
    got = p.double().cpu().numpy().reshape(4, -1).T
    Ki_g = got[:, 0] * got[:, 2] / (got[:, 1] + got[:, 2])
    Ki_t = xi[:, 0] * xi[:, 2] / (xi[:, 1] + xi[:, 2])
    print("median rel err", np.median(np.abs(got - xi) / xi, axis=0))
    assert np.median(np.abs(got - xi) / xi) < 1e-3
    assert np.percentile(np.abs(Ki_g / Ki_t - 1), 95) < 1e-3


def test_fit_writes_model_tacs(cuda_ok):
    import paper_1803_10045_b300 as K
    P, x, maps, lam = _lm_case()
    kin = K.Kinetics(P["ts"], P["te"], S.FENG)
    pg = _t(maps)
    Fo = torch.empty(x.shape, device="cuda")
    K.map_lm_fit(kin, _t(x), pg, 3, 0.1, 0.01, F_out=Fo)
    F_ref = K.tac_eval(kin, pg)
    assert torch.equal(Fo, F_ref)


@pytest.mark.parametrize("delta", [0.01, 1e30])
def test_huber_grad_3d_matches_oracle(cuda_ok, delta):
    import paper_1803_10045_b300 as K
    rng = np.random.default_rng(9)
    maps = rng.uniform(0, 0.1, (4, 5, 13, 11))
    got = K.huber_grad(_t(maps), delta, neighbourhood=26).double().cpu().numpy()
    ref = OL.huber_grad(_f32(maps), delta, nbhd="3d")
    np.testing.assert_allclose(got, ref, atol=4e-6)


@pytest.mark.parametrize("beta", [0.1, 50.0])
def test_single_step_3d_neighbourhood_teacher_forced(cuda_ok, beta):
    """The 26-neighbour (3x3x3) Huber variant: 3 planes of jittered PR1 maps."""
    import paper_1803_10045_b300 as K
    cases = [_lm_case(seed) for seed in (0, 1, 2)]
    P = cases[0][0]
    x = np.concatenate([c[1] for c in cases])
    maps = np.concatenate([c[2] for c in cases], axis=1)
    lam = np.concatenate([c[3] for c in cases])
    kin = K.Kinetics(P["ts"], P["te"], S.FENG)
    pg, lg = _t(maps), _t(lam)
    K.map_lm_fit(kin, _t(x), pg, 1, beta, 0.01, lam=lg, neighbourhood=26)
    got = pg.double().cpu().numpy()
    lam_g = lg.double().cpu().numpy()
    ref, lam_r, acc_r, _ = OL.lm_step(x, maps, lam, P["ts"], P["te"], S.FENG, beta, 0.01,
                                      nbhd="3d")
    acc_g = np.isclose(lam_g, np.maximum(lam / 10, 1e-7), rtol=1e-5)
    agree = acc_g == acc_r
    print(f"3d beta={beta}: accept agreement {agree.mean():.4f}, accepted {acc_r.mean():.3f}")
    assert agree.mean() > 0.99
    tol = 1e-3 * np.maximum(np.abs(ref), FLOOR[:, None, None, None])
    both = agree & np.all(np.abs(got - ref) <= 1e30, axis=0)
    within = np.all(np.abs(got - ref) <= tol, axis=0)[both]
    # the step of a voxel on a flat valley (k2, k3 unidentifiable) amplifies the
    # float32 model error; bound their share, not require it to be zero
    print(f"3d beta={beta}: maps within 1e-3 on {within.mean():.5f} of the voxels")
    assert within.mean() > 0.999
    # the 3D prior couples the planes: the result differs from the in-plane one
    p2 = _t(maps)
    K.map_lm_fit(kin, _t(x), p2, 1, beta, 0.01, lam=_t(lam))
    assert not torch.equal(p2, pg)
