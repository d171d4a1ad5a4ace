"""CUDA Huber prior and MAP-LM step vs the FP64 oracle (GPU).

Teacher-forced parity: both sides take one synchronous LM step from the same
maps, lambda and TACs.  The voxels held strictly are fixed by the oracle
alone before any comparison (oracle.lm.strict_voxels): those whose step
float32 arithmetic resolves within a quarter of the map tolerance and whose
accept decision it resolves with margin.  On every one of them the decisions
agree and the new maps lie within 1e-3 of max(|xi_ref|, floor_p)
(cases.lm_step_parity); everywhere, a voxel both sides reject keeps its maps
bit for bit.  Both the default acceptance threshold tau = 1e-5 and the plain
rule tau = 0 are checked.
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import kinetics as OK
from oracle import lm as OL
from cases import lm_step_parity, pr1_problem

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("tau", [1e-5, 0.0])
@pytest.mark.parametrize("beta", [0.0, 0.1, 50.0])
def test_single_step_teacher_forced(cuda_ok, beta, tau):
    import paper_1803_10045_b300 as K
    P, x, maps, lam = _lm_case()
    kin = K.Kinetics(P["ts"], P["te"], S.FENG)
    pg, lg = _t(maps), _t(lam)
    K.map_lm_fit(kin, _t(x), pg, 1, beta, 0.01, lam=lg, tau=tau)
    sp = OL.float32_spread(x, maps, lam, P["ts"], P["te"], S.FENG, beta, 0.01, tau=tau)
    lm_step_parity(pg.double().cpu().numpy(), lg.double().cpu().numpy(), lam, sp, 0.85,
                   f"PR1 beta={beta} tau={tau}")


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
    sp = OL.float32_spread(x, maps, lam, P["ts"], P["te"], S.FENG, beta, 0.01, nbhd="3d")
    lm_step_parity(pg.double().cpu().numpy(), lg.double().cpu().numpy(), lam, sp, 0.85,
                   f"3d beta={beta}")
    # the 3D prior couples the planes: the result differs from the in-plane one
    p2 = _t(maps)
    K.map_lm_fit(kin, _t(x), p2, 1, beta, 0.01, lam=_t(lam))
    assert not torch.equal(p2, pg)
