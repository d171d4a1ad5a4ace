"""kcs_map_lm_fit_static (GPU): the MAP-LM fit for callers that cannot allocate
device memory -- a host application that owns all device memory through its
own pool and forbids plug-ins to allocate, or a service that must not allocate
after start-up.  Instead of a caller workspace it uses a fixed array inside the
library, so it must give the same maps and model TACs as kcs_map_lm_fit with a
workspace, call after call (the array keeps the previous call's contents).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import kcs_synth as S
from oracle import kinetics as OK

pytestmark = pytest.mark.gpu


def _problem(seed, nz, ny, nx, ts, te):
    """Noisy TACs of jittered parameters and jittered start maps (inputs only)."""
    rng = np.random.default_rng(seed)
    V = nz * ny * nx
    xi = np.clip(S.jittered_params(V, seed=seed, rel=0.4), 0, [2, 2, 1, 1])
    F = OK.model(xi, ts, te, S.FENG, jacobian=False)
    x = (F * (1 + 0.05 * rng.standard_normal(F.shape))).reshape(nz, ny, nx, -1)
    start = (xi * rng.uniform(0.7, 1.3, xi.shape)).T.reshape(4, nz, ny, nx)
    return x, start


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def test_static_scratch_fit_matches_workspace_fit(cuda_ok):
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300._lib import lib
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    kin = K.Kinetics(ts, te, S.FENG)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # calls in a row with different shapes and inputs, with and without a
    # caller lambda: each must not see anything left in the shared array by
    # the one before.  Both paths run the same kernels on the same inputs, so
    # the maps, lambda and model TACs must agree bit for bit.
    cases = [(0, (2, 37, 53), 5, False), (1, (1, 64, 64), 4, True), (2, (3, 11, 9), 6, True)]
    for call, (seed, shape, steps, with_lam) in enumerate(cases):
        nz, ny, nx = shape
        x, start = _problem(seed, nz, ny, nx, ts, te)
        xd = _dev(x)
        pa, pb = _dev(start), _dev(start)
        Fa = torch.empty(x.shape, device="cuda")
        Fb = torch.full(x.shape, float("nan"), device="cuda")
        la = lb = None
        if with_lam:
            lam0 = 10.0 ** np.random.default_rng(seed).uniform(-5, 0, shape)
            la, lb = _dev(lam0), _dev(lam0)
        K.map_lm_fit(kin, xd, pa, steps, 0.1, 0.01, lam=la, F_out=Fa)   # caller workspace
        rc = lib.kcs_map_lm_fit_static(kin.handle, nx, ny, nz, _p(xd), _p(pb), _p(lb), steps,
                                       0.1, 0.01, _p(Fb), stream)
        assert rc == 0, lib.kcs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(pa, pb), call
        assert torch.equal(Fa, Fb), call
        if with_lam:
            assert torch.equal(la, lb), call


def test_static_scratch_rejects_oversize(cuda_ok):
    import paper_1803_10045_b300 as K
    from paper_1803_10045_b300._lib import lib
    ts, te = S.schedule(S.SCHEDULES["pr1"])
    kin = K.Kinetics(ts, te, S.FENG)
    n = 1024   # 1024 x 1024 x 1 voxels > KCS_LM_STATIC_MAX_VOXELS
    rc = lib.kcs_map_lm_fit_static(kin.handle, n, n, 1, C.c_void_p(16), C.c_void_p(16), None, 1,
                                   0.1, 0.01, None, None)
    assert rc == 1
    assert b"at most" in lib.kcs_last_error()
