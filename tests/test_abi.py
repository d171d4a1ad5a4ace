"""Host-side checks of the C ABI: the library loads, exports every declared
symbol, and rejects invalid arguments before touching a GPU (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "kcs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kcs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ["kcs_create_geometry", "kcs_forward_project", "kcs_back_project", "kcs_osl_update",
              "kcs_map_lm_fit", "kcs_icm_iterate"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1803_10045_b300 as K
    lib = C.CDLL(K.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_1803_10045_b300._lib import SIGNATURES
    assert sorted(SIGNATURES) == _declared()


def test_invalid_arguments_are_rejected_on_the_host():
    from paper_1803_10045_b300._lib import lib
    h = C.c_void_p()
    assert lib.kcs_create_geometry(C.byref(h), 0, 4, 1, 2.0, 8, 8, 2.0, 2) == 1
    assert b"positive" in lib.kcs_last_error()
    assert lib.kcs_create_geometry(C.byref(h), 4, 4, 1, 2.0, 8, 8, 2.0, 9) == 1
    assert lib.kcs_forward_project(None, 0, 4, None, None, None) == 1
    assert lib.kcs_osl_update(None, 0, 4, None, 1.0, None, None, 0, None, None, 0.0, 1.0,
                              None, None, 0, None) == 1
    assert lib.kcs_map_lm_fit(None, 4, 4, 1, None, None, None, 1, 0.1, 0.01, None, None, 0,
                              None) == 1
    assert lib.kcs_icm_iterate(None, 1, None) == 1
    assert lib.kcs_icm_iterate_host(None, 1, None, None, 0, None) == 1
    assert lib.kcs_version() >= 1


@pytest.mark.parametrize("M", [3, 36, 0])
def test_frame_count_rule(M):
    from paper_1803_10045_b300._lib import lib
    ts = (C.c_double * max(M, 1))()
    assert lib.kcs_create_kinetics(C.byref(C.c_void_p()), M, ts, ts, ts, None) == 1


def test_workspace_sizes_without_gpu():
    from paper_1803_10045_b300._lib import lib
    assert lib.kcs_lm_workspace_size(10, 10, 2) >= 5 * 200 * 4
    assert lib.kcs_lm_workspace_size(0, 10, 2) == 0
    # ratio row pitch: float rows padded to an odd number of 4-frame quads
    assert [lib.kcs_osl_rho_frames(M, 0) for M in (4, 8, 12, 24, 32)] == [4, 12, 12, 28, 36]
    assert [lib.kcs_osl_rho_frames(M, 1) for M in (4, 8, 24)] == [4, 8, 24]


def test_empty_voxel_sets_need_no_buffers():
    """n_vox = 0 is a no-op for the per-voxel kinetics calls: NULL buffers are
    accepted without touching a device (the kinetics handle is still required)."""
    import ctypes as C
    from paper_1803_10045_b300._lib import lib
    assert lib.kcs_ki(0, None, None, None) == 0
    assert lib.kcs_ki(-1, None, None, None) != 0
    assert lib.kcs_tac_eval(None, 0, None, None, None, None) != 0      # no kinetics handle
