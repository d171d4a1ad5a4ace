"""ctypes loader of libkcs.so and the C signatures of include/kcs.h.

The package has no CPU fallback: if the library is missing the import fails
with instructions to build it.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkcs.so")


class KcsError(RuntimeError):
    """A kcs_* call returned a non-zero status."""

    def __init__(self, status, msg):
        super().__init__(f"kcs status {status}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_1803_10045_b300/build.py` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    return C.CDLL(LIB_PATH)


lib = _load()

vp, i32, i64, f32, sz = C.c_void_p, C.c_int, C.c_int64, C.c_float, C.c_size_t
dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)
pp = C.POINTER(C.c_void_p)


class StudyDesc(C.Structure):
    _fields_ = [("geom", vp), ("kin", vp), ("n_frames", i32), ("kappa", f32), ("frame_dt", vp),
                ("counts", vp), ("randoms", vp), ("randoms_layout", i32), ("bin_factor", vp),
                ("x", vp), ("params", vp), ("F", vp), ("params_given", i32), ("n_lm", i32),
                ("beta_kp", f32), ("sigma2", f32), ("beta_h", f32), ("delta", f32),
                ("workspace", vp), ("ws_bytes", sz), ("counts_type", i32), ("x_type", i32),
                ("x_scale", vp), ("method", i32), ("neighbourhood", i32), ("lm_tau", f32),
                ("lm_tau_given", i32)]


SIGNATURES = {
    "kcs_last_error": (C.c_char_p, []),
    "kcs_version": (i32, []),
    "kcs_create_geometry": (i32, [pp, i32, i32, i32, f32, i32, i32, f32, i32]),
    "kcs_destroy_geometry": (i32, [vp]),
    "kcs_geometry_subset_angles": (i32, [vp, i32, ip, ip]),
    "kcs_forward_project": (i32, [vp, i32, i32, vp, vp, vp]),
    "kcs_back_project": (i32, [vp, i32, i32, vp, vp, vp]),
    "kcs_create_geometry_ex": (i32, [pp, i32, i32, i32, f32, i32, i32, f32, i32, vp]),
    "kcs_forward_project_ex": (i32, [vp, i32, i32, vp, i32, vp, vp, vp]),
    "kcs_back_project_ex": (i32, [vp, i32, i32, vp, i32, vp, vp, vp]),
    "kcs_sensitivity": (i32, [vp, i32, vp, vp, vp]),
    "kcs_osl_workspace_size": (sz, [vp, i32]),
    "kcs_osl_update": (i32, [vp, i32, i32, vp, f32, vp, vp, i32, vp, vp, f32, f32, vp, vp, sz, vp]),
    "kcs_osl_ratio": (i32, [vp, i32, i32, vp, f32, vp, vp, i32, vp, vp, vp, vp]),
    "kcs_osl_backproject": (i32, [vp, i32, i32, vp, f32, vp, vp, vp, f32, f32, vp, vp]),
    "kcs_init_image": (i32, [vp, i32, vp, f32, vp, vp, i32, vp, vp, vp, sz, vp]),
    "kcs_osl_ratio_ex": (i32, [vp, i32, i32, vp, f32, vp, i32, vp, i32, vp, vp, i32, vp, vp, i32,
                               vp]),
    "kcs_osl_backproject_ex": (i32, [vp, i32, i32, vp, f32, vp, vp, i32, vp, f32, f32, vp, i32, vp,
                                     vp]),
    "kcs_osl_rho_frames": (i32, [i32, i32]),
    "kcs_osl_update_ex": (i32, [vp, i32, i32, vp, f32, vp, i32, vp, i32, vp, vp, f32, f32, vp, i32,
                                vp, vp, sz, vp]),
    "kcs_loglik": (i32, [vp, i32, vp, f32, vp, i32, vp, i32, vp, vp, i32, vp, vp, vp, sz, vp]),
    "kcs_init_level": (i32, [vp, i32, vp, f32, vp, i32, vp, i32, vp, vp, vp, sz, vp]),
    "kcs_init_image_ex": (i32, [vp, i32, vp, f32, vp, i32, vp, i32, vp, vp, i32, vp, vp, sz, vp]),
    "kcs_huber_grad_nb": (i32, [i32, i32, i32, vp, f32, i32, vp, vp]),
    "kcs_map_lm_fit_nb": (i32, [vp, i32, i32, i32, vp, i32, vp, vp, vp, i32, f32, f32, i32, f32,
                                vp, vp, sz, vp]),
    "kcs_map_lm_fit_ex": (i32, [vp, i32, i32, i32, vp, i32, vp, vp, vp, i32, f32, f32, vp, vp, sz,
                                vp]),
    "kcs_create_kinetics": (i32, [pp, i32, dp, dp, dp, vp]),
    "kcs_destroy_kinetics": (i32, [vp]),
    "kcs_tac_eval": (i32, [vp, i64, vp, vp, vp, vp]),
    "kcs_ki": (i32, [i64, vp, vp, vp]),
    "kcs_tac_vjp": (i32, [vp, i64, vp, vp, vp, vp]),
    "kcs_huber_grad": (i32, [i32, i32, i32, vp, f32, vp, vp]),
    "kcs_lm_workspace_size": (sz, [i32, i32, i32]),
    "kcs_map_lm_fit": (i32, [vp, i32, i32, i32, vp, vp, vp, i32, f32, f32, vp, vp, sz, vp]),
    "kcs_map_lm_fit_static": (i32, [vp, i32, i32, i32, vp, vp, vp, i32, f32, f32, vp, vp]),
    "kcs_study_workspace_size": (sz, [vp, i32]),
    "kcs_create_study": (i32, [pp, C.POINTER(StudyDesc)]),
    "kcs_destroy_study": (i32, [vp]),
    "kcs_icm_iterate": (i32, [vp, i32, vp]),
    "kcs_icm_iterate_host": (i32, [vp, i32, vp, vp, sz, vp]),
    "kcs_study_iterations": (i32, [vp]),
    "kcs_study_set_iterations": (i32, [vp, i32]),
    "kcs_study_set_graph": (i32, [vp, i32]),
    "kcs_study_fit": (i32, [vp, i32, vp]),
    "kcs_device_status": (i32, [C.POINTER(C.c_uint)]),
    "kcs_device_status_reset": (i32, []),
    "kcs_selftest_wait_timeout": (i32, [i32, vp]),
    "kcs_fma_peak_launch": (i32, [i32, i32, i32, dp, vp, vp]),
}

for _name, (_res, _args) in SIGNATURES.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def check(status):
    """Raise KcsError with the library's message for a non-zero status."""
    if status != 0:
        raise KcsError(status, lib.kcs_last_error().decode())
    return status
