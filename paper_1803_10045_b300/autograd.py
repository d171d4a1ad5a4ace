"""Differentiable forward model y = P F(theta) (torch.autograd.Function).

forward:  F = kcs_tac_eval(theta) (frame-integrated FDG two-tissue model), then
          y = kcs_forward_project(F) on the rays of one subset or all angles.
backward: g_F = kcs_back_project(g_y) (the exact transpose), then
          g_theta = kcs_tac_vjp(theta, g_F) (the analytic kinetic Jacobian
          transposed).  Both steps are the library's kernels.

A batch of studies with the same geometry and frame schedule is passed as
theta [B][4][Z][Y][X]; planes are independent, so the batch is folded into the
plane axis of a geometry with B*Z planes.
"""
from __future__ import annotations

import torch

from . import api
from ._lib import check, lib


def tac_vjp(kin: api.Kinetics, params, gF):
    """gparams [4][...] = J^T gF per voxel (params [4][...], gF [...][M])."""
    shp = tuple(params.shape[1:])
    out = torch.empty_like(params)
    n = out[0].numel()
    check(lib.kcs_tac_vjp(kin.handle, n, api._ptr(params, "params"),
                          api._ptr(gF, "gF", shp + (kin.M,)), api._ptr(out, "gparams"),
                          api._stream()))
    return out


class KineticForward(torch.autograd.Function):
    """y [Z][A_k][B][M] = P_k F(params [4][Z][Y][X]); differentiable in params."""

    @staticmethod
    def forward(ctx, params, geom, kin, subset=-1):
        params = params.contiguous()
        F = api.tac_eval(kin, params)
        y = api.forward_project(geom, F, subset)
        ctx.save_for_backward(params)
        ctx.geom, ctx.kin, ctx.subset = geom, kin, subset
        return y

    @staticmethod
    def backward(ctx, gy):
        (params,) = ctx.saved_tensors
        gF = api.back_project(ctx.geom, gy.contiguous(), ctx.subset)
        return tac_vjp(ctx.kin, params, gF), None, None, None


def forward_model(theta, geom, kin, subset=-1):
    """y = P F(theta) for theta [4][Z][Y][X] or a batch [B][4][Z][Y][X]
    (geometry with B*Z planes); returns [Z][A_k][B][M] or [B][Z][A_k][B][M]."""
    if theta.dim() == 4:
        return KineticForward.apply(theta, geom, kin, subset)
    B, _, Z, Y, X = theta.shape
    folded = theta.permute(1, 0, 2, 3, 4).reshape(4, B * Z, Y, X)
    y = KineticForward.apply(folded, geom, kin, subset)
    return y.reshape(B, Z, *y.shape[1:])
