"""Thin torch-facing wrappers of the kcs C ABI (argument marshalling only).

Every array is a CUDA float32 tensor in the layout the C header states; the
wrappers check device, dtype, shape and contiguity, pass raw pointers and the
current torch stream, and raise KcsError on a non-zero status.  All arithmetic
runs in libkcs.so's kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from ._lib import StudyDesc, check, lib

RANDOMS_NONE, RANDOMS_PER_FRAME, RANDOMS_FULL = 0, 1, 2
F32, BF16, F16, U16 = 0, 1, 2, 3
METHODS = {"kcs": 0, "direct": 1, "indirect": 2}
_STORAGE = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16, torch.uint16: U16}


def _storage(t, allowed, name):
    code = _STORAGE.get(t.dtype)
    if code not in allowed:
        raise ValueError(f"{name} has unsupported dtype {t.dtype}")
    return code


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, name, shape=None, dtype=torch.float32, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


class Geometry:
    """Parallel-beam stacked-2D Joseph geometry with S ordered subsets."""

    def __init__(self, nx, ny, nz, vox_mm, n_bins, n_angles, bin_mm, n_subsets):
        h = C.c_void_p()
        # synchronous: the geometry may be used from any stream afterwards
        check(lib.kcs_create_geometry(C.byref(h), nx, ny, nz, vox_mm, n_bins, n_angles, bin_mm,
                                      n_subsets))
        self.handle = h
        self.nx, self.ny, self.nz = nx, ny, nz
        self.vox_mm, self.bin_mm = vox_mm, bin_mm
        self.n_bins, self.n_angles, self.n_subsets = n_bins, n_angles, n_subsets
        self._sub = {}

    def subset_angles(self, k):
        if k not in self._sub:
            n = C.c_int()
            check(lib.kcs_geometry_subset_angles(self.handle, k, None, C.byref(n)))
            out = (C.c_int * n.value)()
            check(lib.kcs_geometry_subset_angles(self.handle, k, out, C.byref(n)))
            self._sub[k] = np.array(out[:], dtype=np.int64)
        return self._sub[k]

    def n_sub(self, k):
        return len(self.subset_angles(k))

    def image_shape(self, M):
        return (self.nz, self.ny, self.nx, M)

    def sino_shape(self, M, k=-1):
        return (self.nz, self.n_angles if k < 0 else self.n_sub(k), self.n_bins, M)

    def close(self):
        if getattr(self, "handle", None):
            lib.kcs_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def forward_project(g: Geometry, x, subset=-1, out=None, x_scale=None):
    """y = P_k x for every frame: [Z][ny][nx][M] -> [Z][A_k][B][M] (float32).
    x float32, or bfloat16 / float16 holding x / x_scale[m]."""
    M = x.shape[-1]
    xt = _storage(x, (F32, BF16, F16), "x")
    px = _ptr(x, "x", g.image_shape(M), dtype=x.dtype)
    if out is None:
        out = torch.empty(g.sino_shape(M, subset), device=x.device, dtype=torch.float32)
    py = _ptr(out, "out", g.sino_shape(M, subset))
    if xt == F32 and x_scale is None:
        check(lib.kcs_forward_project(g.handle, subset, M, px, py, _stream()))
    else:
        check(lib.kcs_forward_project_ex(g.handle, subset, M, px, xt,
                                         _ptr(x_scale, "x_scale", (M,), allow_none=True), py,
                                         _stream()))
    return out


def back_project(g: Geometry, y, subset=-1, out=None, y_scale=None):
    """x = P_k^T y for every frame: [Z][A_k][B][M] -> [Z][ny][nx][M] (float32).
    y float32, or bfloat16 / float16 holding y / y_scale[m]."""
    M = y.shape[-1]
    yt = _storage(y, (F32, BF16, F16), "y")
    py = _ptr(y, "y", g.sino_shape(M, subset), dtype=y.dtype)
    if out is None:
        out = torch.empty(g.image_shape(M), device=y.device, dtype=torch.float32)
    px = _ptr(out, "out", g.image_shape(M))
    if yt == F32 and y_scale is None:
        check(lib.kcs_back_project(g.handle, subset, M, py, px, _stream()))
    else:
        check(lib.kcs_back_project_ex(g.handle, subset, M, py, yt,
                                      _ptr(y_scale, "y_scale", (M,), allow_none=True), px,
                                      _stream()))
    return out


def sensitivity(g: Geometry, subset=-1, bin_factor=None, device="cuda"):
    out = torch.empty((g.nz, g.ny, g.nx), device=device, dtype=torch.float32)
    pb = _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True)
    check(lib.kcs_sensitivity(g.handle, subset, pb, _ptr(out, "sens"), _stream()))
    return out


def _randoms(g, randoms, M):
    if randoms is None:
        return None, RANDOMS_NONE
    if randoms.dim() == 1:
        return _ptr(randoms, "randoms", (M,)), RANDOMS_PER_FRAME
    return _ptr(randoms, "randoms", g.sino_shape(M)), RANDOMS_FULL


def device_status():
    """Bounded in-kernel waits that ran out on the current device (0 = none)."""
    n = C.c_uint(0)
    rc = lib.kcs_device_status(C.byref(n))
    if rc not in (0, 4):
        check(rc)
    return n.value


def osl_workspace_size(g: Geometry, M):
    return lib.kcs_osl_workspace_size(g.handle, M)


def osl_update(g: Geometry, subset, x, frame_dt, kappa, counts, randoms=None, bin_factor=None,
               F=None, beta=0.0, sigma2=1.0, workspace=None, x_scale=None):
    """One OS-MAP-OSL-KP update of x (in place) on subset k.  x may be float32,
    bfloat16 or float16 (stored x / x_scale[m]); counts float32 or uint16."""
    M = x.shape[-1]
    pr, layout = _randoms(g, randoms, M)
    xt = _storage(x, (F32, BF16, F16), "x")
    ct = _storage(counts, (F32, U16), "counts")
    if workspace is None:
        workspace = _workspace(osl_workspace_size(g, M), x.device)
    check(lib.kcs_osl_update_ex(
        g.handle, subset, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(counts, "counts", g.sino_shape(M), dtype=counts.dtype), ct, pr, layout,
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(F, "F", g.image_shape(M), allow_none=True), float(beta), float(sigma2),
        _ptr(x, "x", g.image_shape(M), dtype=x.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True), C.c_void_p(workspace.data_ptr()),
        workspace.numel(), _stream()))
    return x


def rho_frames(M, dtype=torch.float32):
    """Row pitch (frames) of the ratio rows that osl_update keeps internally and
    that osl_ratio allocates by default: M padded to an odd number of 4-frame
    quads for float32, M for 16-bit storage."""
    return lib.kcs_osl_rho_frames(int(M), _STORAGE.get(dtype, F32))


def osl_ratio(g: Geometry, subset, x, frame_dt, kappa, counts, randoms=None, bin_factor=None,
              out=None, x_scale=None):
    """rho = s / ybar on the rays of subset k, stored in x's dtype (float32,
    bfloat16 or float16; x holds x / x_scale[m]): out [Z][A_k][B][P] with the
    ratio in frames [..., :M]; P = rho_frames(M, dtype) by default, or out's
    own last dimension (a multiple of 4, >= M; M gives dense rows)."""
    M = x.shape[-1]
    pr, layout = _randoms(g, randoms, M)
    xt = _storage(x, (F32, BF16, F16), "x")
    ct = _storage(counts, (F32, U16), "counts")
    if out is None:
        out = torch.empty(g.sino_shape(rho_frames(M, x.dtype), subset), device=x.device,
                          dtype=x.dtype)
    P = out.shape[-1]
    check(lib.kcs_osl_ratio_ex(
        g.handle, subset, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(counts, "counts", g.sino_shape(M), dtype=counts.dtype), ct, pr, layout,
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(x, "x", g.image_shape(M), dtype=x.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True),
        _ptr(out, "rho", g.sino_shape(P, subset), dtype=x.dtype), P, _stream()))
    return out


def osl_backproject(g: Geometry, subset, x, frame_dt, kappa, rho, bin_factor=None, F=None,
                    beta=0.0, sigma2=1.0, x_scale=None):
    """OSL update of x (in place) from a ratio sinogram rho of subset k (rho in
    x's dtype, [Z][A_k][B][P] with the ratio in frames [..., :M], as osl_ratio
    writes it)."""
    M = x.shape[-1]
    xt = _storage(x, (F32, BF16, F16), "x")
    P = rho.shape[-1]
    check(lib.kcs_osl_backproject_ex(
        g.handle, subset, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(rho, "rho", g.sino_shape(P, subset), dtype=x.dtype), P,
        _ptr(F, "F", g.image_shape(M), allow_none=True), float(beta), float(sigma2),
        _ptr(x, "x", g.image_shape(M), dtype=x.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True), _stream()))
    return x


def loglik(g: Geometry, x, frame_dt, kappa, counts, randoms=None, bin_factor=None,
           x_scale=None, workspace=None):
    """Poisson log-likelihood sum s log ybar - ybar of image x (a 0-d float64
    CUDA tensor; one full forward projection)."""
    M = x.shape[-1]
    pr, layout = _randoms(g, randoms, M)
    xt = _storage(x, (F32, BF16, F16), "x")
    ct = _storage(counts, (F32, U16), "counts")
    out = torch.empty((), device=x.device, dtype=torch.float64)
    if workspace is None:
        workspace = _workspace(8192, x.device)
    check(lib.kcs_loglik(
        g.handle, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(counts, "counts", g.sino_shape(M), dtype=counts.dtype), ct, pr, layout,
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(x, "x", g.image_shape(M), dtype=x.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True),
        C.c_void_p(out.data_ptr()), C.c_void_p(workspace.data_ptr()), workspace.numel(),
        _stream()))
    return out


def init_level(g: Geometry, frame_dt, kappa, counts, randoms=None, bin_factor=None,
               workspace=None, out=None):
    """Per-frame level c_m [M] of the uniform start image (the precision form's
    natural per-frame scale)."""
    M = counts.shape[-1]
    pr, layout = _randoms(g, randoms, M)
    ct = _storage(counts, (F32, U16), "counts")
    if out is None:
        out = torch.empty(M, device=counts.device, dtype=torch.float32)
    if workspace is None:
        workspace = _workspace(osl_workspace_size(g, M), counts.device)
    check(lib.kcs_init_level(
        g.handle, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(counts, "counts", g.sino_shape(M), dtype=counts.dtype), ct, pr, layout,
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(out, "level", (M,)), C.c_void_p(workspace.data_ptr()), workspace.numel(), _stream()))
    return out


def init_image(g: Geometry, frame_dt, kappa, counts, randoms=None, bin_factor=None, out=None,
               workspace=None, dtype=torch.float32, x_scale=None):
    """Uniform per-frame start image matching the measured trues (stored as
    dtype holding c_m / x_scale[m])."""
    M = counts.shape[-1]
    pr, layout = _randoms(g, randoms, M)
    if out is None:
        out = torch.empty(g.image_shape(M), device=counts.device, dtype=dtype)
    xt = _storage(out, (F32, BF16, F16), "out")
    ct = _storage(counts, (F32, U16), "counts")
    if workspace is None:
        workspace = _workspace(osl_workspace_size(g, M), counts.device)
    check(lib.kcs_init_image_ex(
        g.handle, M, _ptr(frame_dt, "frame_dt", (M,)), float(kappa),
        _ptr(counts, "counts", g.sino_shape(M), dtype=counts.dtype), ct, pr, layout,
        _ptr(bin_factor, "bin_factor", (g.nz, g.n_angles, g.n_bins), allow_none=True),
        _ptr(out, "out", g.image_shape(M), dtype=out.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True), C.c_void_p(workspace.data_ptr()),
        workspace.numel(), _stream()))
    return out


class Kinetics:
    """Frame schedule + Feng input; tabulates the model's series coefficients."""

    def __init__(self, t_start, t_end, feng):
        ts = np.ascontiguousarray(t_start, dtype=np.float64)
        te = np.ascontiguousarray(t_end, dtype=np.float64)
        fe = np.array([feng["A1"], feng["A2"], feng["A3"], feng["l1"], feng["l2"], feng["l3"]],
                      dtype=np.float64)
        h = C.c_void_p()
        dptr = C.POINTER(C.c_double)
        check(lib.kcs_create_kinetics(C.byref(h), len(ts), ts.ctypes.data_as(dptr),
                                      te.ctypes.data_as(dptr), fe.ctypes.data_as(dptr), _stream()))
        self.handle = h
        self.M = len(ts)
        self.t_start, self.t_end = ts, te

    def close(self):
        if getattr(self, "handle", None):
            lib.kcs_destroy_kinetics(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def tac_eval(kin: Kinetics, params, jacobian=False, out=None):
    """params [4][...] -> F [...][M] (and J [...][M][4])."""
    shp = tuple(params.shape[1:])
    n = int(np.prod(shp)) if shp else 1
    F = out if out is not None else torch.empty(shp + (kin.M,), device=params.device,
                                                dtype=torch.float32)
    J = torch.empty(shp + (kin.M, 4), device=params.device, dtype=torch.float32) if jacobian else None
    check(lib.kcs_tac_eval(kin.handle, n, _ptr(params, "params"), _ptr(F, "F", shp + (kin.M,)),
                           _ptr(J, "J", allow_none=True), _stream()))
    return (F, J) if jacobian else F


def ki(params):
    """Ki = K1 k3 / (k2 + k3) per voxel."""
    shp = tuple(params.shape[1:])
    out = torch.empty(shp, device=params.device, dtype=torch.float32)
    check(lib.kcs_ki(out.numel(), _ptr(params, "params"), _ptr(out, "ki"), _stream()))
    return out


def huber_grad(params, delta, neighbourhood=8):
    """dH/dxi of maps [4][Z][Y][X] over 8 in-plane or 26 (3x3x3) neighbours."""
    _, nz, ny, nx = params.shape
    out = torch.empty_like(params)
    check(lib.kcs_huber_grad_nb(nx, ny, nz, _ptr(params, "params"), float(delta),
                                int(neighbourhood), _ptr(out, "grad"), _stream()))
    return out


def lm_workspace_size(nx, ny, nz):
    return lib.kcs_lm_workspace_size(nx, ny, nz)


LM_TAU_DEFAULT = 1e-5   # KCS_LM_TAU_DEFAULT of kcs.h


def map_lm_fit(kin: Kinetics, x, params, n_steps, beta_h, delta, lam=None, F_out=None,
               workspace=None, x_scale=None, neighbourhood=8, tau=LM_TAU_DEFAULT):
    """n_steps MAP-LM steps on params [4][Z][Y][X] (in place) for TACs x [Z][Y][X][M]
    (x float32, bfloat16 or float16 holding x / x_scale[m]); a trial is accepted
    when it lowers the voxel objective by more than tau of its value."""
    nz, ny, nx, M = x.shape
    xt = _storage(x, (F32, BF16, F16), "x")
    if workspace is None:
        workspace = _workspace(lm_workspace_size(nx, ny, nz), x.device)
    check(lib.kcs_map_lm_fit_nb(
        kin.handle, nx, ny, nz, _ptr(x, "x", (nz, ny, nx, M), dtype=x.dtype), xt,
        _ptr(x_scale, "x_scale", (M,), allow_none=True), _ptr(params, "params", (4, nz, ny, nx)),
        _ptr(lam, "lambda", (nz, ny, nx), allow_none=True), int(n_steps), float(beta_h), float(delta),
        int(neighbourhood), float(tau), _ptr(F_out, "F_out", (nz, ny, nx, M), allow_none=True),
        C.c_void_p(workspace.data_ptr()), workspace.numel(), _stream()))
    return params


class Study:
    """Device-resident ICM state of one dynamic study (caller-owned tensors)."""

    def __init__(self, geom: Geometry, kin: Kinetics, frame_dt, kappa, counts, x, params, F=None,
                 randoms=None, bin_factor=None, params_given=False, n_lm=10, beta_kp=0.1,
                 sigma2=1.0, beta_h=0.1, delta=0.01, workspace=None, x_scale=None, graph=False,
                 method="kcs", neighbourhood=8, tau=LM_TAU_DEFAULT):
        M = kin.M
        dev = x.device
        if F is None:
            F = torch.zeros(geom.image_shape(M), device=dev, dtype=torch.float32)
        if workspace is None:
            workspace = _workspace(lib.kcs_study_workspace_size(geom.handle, M), dev)
        pr, layout = _randoms(geom, randoms, M)
        self._keep = (geom, kin, frame_dt, counts, x, params, F, randoms, bin_factor, workspace,
                      x_scale)
        self.geom, self.kin, self.x, self.params, self.F = geom, kin, x, params, F
        self.kappa = float(kappa)
        d = StudyDesc()
        d.geom, d.kin, d.n_frames, d.kappa = geom.handle, kin.handle, M, float(kappa)
        d.frame_dt = _ptr(frame_dt, "frame_dt", (M,))
        d.counts = _ptr(counts, "counts", geom.sino_shape(M), dtype=counts.dtype)
        d.counts_type = _storage(counts, (F32, U16), "counts")
        d.x_type = _storage(x, (F32, BF16, F16), "x")
        d.x_scale = _ptr(x_scale, "x_scale", (M,), allow_none=True)
        d.randoms, d.randoms_layout = pr, layout
        d.bin_factor = _ptr(bin_factor, "bin_factor", (geom.nz, geom.n_angles, geom.n_bins),
                            allow_none=True)
        d.x = _ptr(x, "x", geom.image_shape(M), dtype=x.dtype)
        d.params = _ptr(params, "params", (4, geom.nz, geom.ny, geom.nx))
        d.F = _ptr(F, "F", geom.image_shape(M))
        d.params_given, d.n_lm = int(bool(params_given)), int(n_lm)
        d.beta_kp, d.sigma2, d.beta_h, d.delta = float(beta_kp), float(sigma2), float(beta_h), float(delta)
        d.workspace, d.ws_bytes = C.c_void_p(workspace.data_ptr()), workspace.numel()
        if method not in METHODS:
            raise ValueError(f"method must be one of {sorted(METHODS)}")
        d.method = METHODS[method]
        d.neighbourhood = int(neighbourhood)
        d.lm_tau, d.lm_tau_given = float(tau), 1
        h = C.c_void_p()
        check(lib.kcs_create_study(C.byref(h), C.byref(d)))
        self.handle = h
        if graph:
            self.set_graph(True)

    def set_graph(self, enable=True):
        """Replay the steady-state ICM iteration from a CUDA graph."""
        check(lib.kcs_study_set_graph(self.handle, int(bool(enable))))

    def iterate(self, n_iter=1):
        check(lib.kcs_icm_iterate(self.handle, int(n_iter), _stream()))

    def iterate_host(self, n_iter, counts_host=None, params_host=None):
        """n_iter ICM iterations streaming host data: the counts are copied in
        from counts_host (pinned, the study's counts shape and dtype) before
        every iteration and the maps copied out to params_host after every
        iteration (pinned float32, [4][Z][ny][nx] overwritten each time, or
        [n_iter][4][Z][ny][nx] for one set per iteration).  The copies overlap
        the compute; results equal iterate's.  Asynchronous on the current
        stream; keep the host tensors alive until it completes."""
        g = self.geom
        counts = self._keep[3]
        pc = pp = None
        stride = 0
        if counts_host is not None:
            if (counts_host.device.type != "cpu" or not counts_host.is_pinned()
                    or counts_host.dtype != counts.dtype or counts_host.shape != counts.shape
                    or not counts_host.is_contiguous()):
                raise ValueError("counts_host must be pinned, contiguous and shaped like the counts")
            pc = C.c_void_p(counts_host.data_ptr())
        if params_host is not None:
            shape = (4, g.nz, g.ny, g.nx)
            if params_host.dim() == 5:
                if tuple(params_host.shape) != (n_iter,) + shape:
                    raise ValueError(f"params_host must be {(n_iter,) + shape} or {shape}")
                stride = params_host[0].numel()
            elif tuple(params_host.shape) != shape:
                raise ValueError(f"params_host must be {shape} or {(n_iter,) + shape}")
            if (params_host.device.type != "cpu" or not params_host.is_pinned()
                    or params_host.dtype != torch.float32 or not params_host.is_contiguous()):
                raise ValueError("params_host must be pinned, contiguous float32")
            pp = C.c_void_p(params_host.data_ptr())
        check(lib.kcs_icm_iterate_host(self.handle, int(n_iter), pc, pp, stride, _stream()))

    def loglik(self):
        """Poisson log-likelihood of the current image (0-d float64 tensor)."""
        g, kin, frame_dt, counts, x, params, F, randoms, bin_factor, workspace, x_scale = self._keep
        return loglik(g, x, frame_dt, self.kappa, counts, randoms, bin_factor, x_scale,
                      workspace)

    def fit(self, n_steps):
        """Post-reconstruction kinetic fit of the current image (INDIRECT)."""
        check(lib.kcs_study_fit(self.handle, int(n_steps), _stream()))

    @property
    def iterations(self):
        return lib.kcs_study_iterations(self.handle)

    def save(self, path):
        """Checkpoint the ICM state (image series, kinetic maps, model TACs,
        iteration count) to an .npz file; arrays keep their storage dtype's
        bits.  Synchronises the current stream."""
        import numpy as np
        torch.cuda.current_stream().synchronize()

        def host(t):
            if t.dtype in (torch.bfloat16, torch.float16):
                return t.view(torch.int16).cpu().numpy(), str(t.dtype)
            return t.cpu().numpy(), str(t.dtype)
        x, xd = host(self.x)
        np.savez(path, x=x, x_dtype=xd, params=self.params.cpu().numpy(),
                 F=self.F.cpu().numpy(), iterations=self.iterations)

    def restore(self, path):
        """Load a checkpoint written by save into this study's buffers (same
        shapes and storage types) and resume its iteration count."""
        import numpy as np
        d = np.load(path)
        if str(d["x_dtype"]) != str(self.x.dtype):
            raise ValueError(f"checkpoint holds {d['x_dtype']}, study x is {self.x.dtype}")
        x = torch.from_numpy(d["x"])
        if self.x.dtype in (torch.bfloat16, torch.float16):
            x = x.view(self.x.dtype)
        self.x.copy_(x)
        self.params.copy_(torch.from_numpy(d["params"]))
        self.F.copy_(torch.from_numpy(d["F"]))
        check(lib.kcs_study_set_iterations(self.handle, int(d["iterations"])))

    def close(self):
        if getattr(self, "handle", None):
            lib.kcs_destroy_study(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
