"""B300-native hot path of Kinetic Compressive Sensing (Scipioni et al.).

The ICM loop of direct parametric PET reconstruction -- OS-MAP-OSL image
updates with a kinetics-derived prior and a voxel-parallel MAP
Levenberg-Marquardt fit of the FDG two-tissue model under a Huber MRF prior --
as hand-written sm_103a CUDA kernels behind the C ABI of include/kcs.h
(libkcs.so).  This package is the thin Python binding: it marshals torch CUDA
tensors into that ABI and has no CPU fallback.  Around it: the differentiable
forward model (autograd), a serving loop for many studies under an HBM budget
(serving), and plane sharding across ranks (sharding).
"""
from ._lib import LIB_PATH, KcsError, lib  # noqa: F401
from .api import (  # noqa: F401
    RANDOMS_FULL, RANDOMS_NONE, RANDOMS_PER_FRAME, Geometry, Kinetics, Study, back_project,
    device_status,
    forward_project, huber_grad, init_image, init_level, ki, loglik, lm_workspace_size, map_lm_fit, osl_backproject,
    osl_ratio, osl_update, osl_workspace_size, rho_frames, sensitivity, tac_eval)
from .autograd import KineticForward, forward_model, tac_vjp  # noqa: F401,E402
