"""CUDA frame-integrated 2TC model (F and Jacobian) vs the FP64 oracle (GPU).

Tolerance derivation: the kernel evaluates per-cell cubic Hermite
interpolants of a float64 table of the frame averages (a = k2 + k3, spacing
1/512), with the coefficients and a handful of fused multiply-adds in float32.
A CPU emulation of that table against the exact model puts the values within
2.3e-7 of each voxel's largest |F| and the derivative columns within 3.1e-6 of
each column's largest entry (the slopes carry the cubic's truncation).  The
tests hold F to 1e-6 of the voxel's largest |F| and every Jacobian entry to
2e-5 of the voxel's largest Jacobian entry (dF/dk3 = -(1-Vb) K1 k2 B' is
exactly 0 at k2 = 0, so it is measured against the row, not its own column).
"""
import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import kinetics as OK

pytestmark = pytest.mark.gpu

L3, L2 = S.FENG["l3"], S.FENG["l2"]
EDGE = np.array([
    [0.10, 0.13, 0.06, 0.04],      # GM
    [0.05, 0.10, 0.04, 0.03],      # WM
    [0.03, 0.08, 0.02, 0.02],      # background
    [0.30, 0.0, 0.0, 0.05],        # a = 0
    [0.30, 1e-7, 1e-7, 0.05],      # a -> 0
    [0.20, L3 - 0.05, 0.05, 0.1],  # a = l3
    [0.20, L2, 0.0, 0.1],          # a = l2
    [2.0, 2.0, 1.0, 0.0],          # upper corner of the LM box
    [0.0, 0.5, 0.5, 0.3],          # K1 = 0
    [0.4, 0.2, 0.1, 1.0],          # pure blood
    [1.0, 0.01, 0.99, 0.5],
    [0.2, 0.3 - 1e-6, 0.0, 0.05],  # a just below a table node (t -> 1)
    [0.2, 0.3125, 0.0, 0.05],      # a exactly on a node (t = 0)
    [0.5, 2.0, 1.0, 0.05],         # a = 3, the box maximum
    [0.5, 2.7, 1.0, 0.05],         # a = 3.7, near the end of the table
])

SCHEDS = {
    "pr1": S.schedule(S.SCHEDULES["pr1"]),
    "pr2": S.schedule(S.SCHEDULES["pr2"]),
    "paper": S.schedule(S.SCHEDULES["paper"]),          # 600 s frame: split on the device
    "gaps": (np.array([0.5, 1.0, 4.0, 10.0]), np.array([0.75, 2.0, 7.0, 12.5])),
    "m32": S.schedule([(8, 10), (8, 30), (8, 120), (8, 300)]),   # the maximum of 32 frames
}


def _check(ts, te, xi):
    import paper_1803_10045_b300 as K
    kin = K.Kinetics(ts, te, S.FENG)
    p = torch.tensor(xi.T.copy(), dtype=torch.float32, device="cuda")
    F, J = K.tac_eval(kin, p, jacobian=True)
    F = F.double().cpu().numpy()
    J = J.double().cpu().numpy()
    # the oracle sees the parameters the GPU saw (float32-rounded)
    Fr, Jr = OK.model(xi.astype(np.float32).astype(np.float64), ts, te, S.FENG)
    eF = np.abs(F - Fr).max(axis=1) / np.abs(Fr).max(axis=1).clip(1e-30)
    row = np.abs(Jr).max(axis=(1, 2)) + 1e-30
    eJ = np.abs(J - Jr).max(axis=1) / row[:, None]
    print(f"max |dF| / max|F| {eF.max():.2e}; max |dJ_q| / max|J| "
          + " ".join(f"{eJ[:, q].max():.2e}" for q in range(4)))
    assert eF.max() < 1e-6
    assert eJ.max() < 2e-5


@pytest.mark.parametrize("sched", list(SCHEDS))
def test_model_edge_cases(cuda_ok, sched):
    ts, te = SCHEDS[sched]
    _check(ts, te, EDGE)


@pytest.mark.parametrize("sched", ["pr1", "pr2"])
def test_model_jittered(cuda_ok, sched):
    ts, te = SCHEDS[sched]
    xi = np.clip(S.jittered_params(3000, seed=9, rel=0.9), 0, [2, 2, 1, 1])
    _check(ts, te, xi)


def test_ki(cuda_ok):
    import paper_1803_10045_b300 as K
    p = torch.tensor(EDGE.T.copy(), dtype=torch.float32, device="cuda")
    got = K.ki(p).double().cpu().numpy()
    np.testing.assert_allclose(got, OK.ki(EDGE.T.astype(np.float32).astype(np.float64)), rtol=1e-6)


def test_empty_voxel_set_is_a_no_op(cuda_ok):
    import paper_1803_10045_b300 as K
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    kin = K.Kinetics(ts, te, S.FENG)
    p = torch.empty((4, 0), device="cuda")
    F, J = K.tac_eval(kin, p, jacobian=True)
    torch.cuda.synchronize()
    assert F.shape == (0, 12) and J.shape == (0, 12, 4)
