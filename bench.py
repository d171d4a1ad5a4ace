#!/usr/bin/env python
"""ICM throughput on the full-size stacked-2D workload (one JSON line).

Workload (config PR2): 344 x 344 x 127 voxels of 2.09 mm, 24 frames (8x15 s,
4x60 s, 6x180 s, 6x300 s), 344 bins x 252 angles, 21 subsets, brain-like
phantom with 20 lesions and 10 % parameter jitter, ~2e8 prompts (80 % trues,
20 % uniform randoms), 10 MAP-LM steps per ICM iteration.  A step is one ICM
iteration: 21 x (forward projection + ratio, back-projection + OSL update),
10 MAP-LM steps and the model TACs for the next prior.  Inputs are synthetic
(the paper's human data are not available) and resident in HBM; the image
series (1.44 GB) and the counts (1.06 GB) are larger than the 126 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--storage f32|bf16|f16]

--storage bf16 / f16 runs the precision form: image series and ratio
sinograms stored in bfloat16 / float16 with a per-frame scale (max of the start
image); arithmetic stays float32.  The default is float32.  The measured
counts are integers and are held as uint16 by default (exact; --counts f32
for float32 counts, bit-identical results).

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one plane, one subset update, one LM step on 4096 voxels) and
extrapolates to ICM iter/s; it is a deliberately slow, untuned baseline.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import kcs_synth as S  # noqa: E402

METRIC = "ICM iter/s at 344²×127×24 frames"
WORKLOAD = "PR2: 344x344x127 (2.09 mm), 344 bins x 252 angles, 24 frames, 21 subsets, 10 LM steps/iter"
N_LM = 10
BETA_H, DELTA = 0.1, 0.01
# The kinetics-derived prior competes with kappa dt sens in the OSL denominator,
# so its weight scales with the count calibration.  Linearised at x = F, one
# OSL update multiplies a deviation x - F by 1 - r with
# r = beta_kp F / (S sigma2 kappa dt sens): the update is stable only for
# r < 2, and the short early frames of PR2 at its hottest voxels reached
# r = 2.3 with beta_kp = 0.1 kappa / kappa_PR1.  beta_kp = 0.01 kappa /
# kappa_PR1 (the prior-to-data ratio of the end-to-end parity tests' stable
# weight on config PR1, beta_kp = 0.01 at kappa ~ 5e-3) keeps r below 0.25.
KAPPA_PR1 = 5.06e-3


def beta_kp_for(kappa):
    return 0.01 * kappa / KAPPA_PR1
FP32_LANES_PER_SM, N_SM = 128, 148


def lm_flops_per_voxel_step(frames=24, n_lm=10):
    """Nominal float32 flops (FMA = 2) of one MAP-LM voxel-step: one model +
    Jacobian evaluation at the trial point (the current point's normal
    equations are kept from the previous step): per frame the cell cubics of
    A, B and their slopes (10 FMA), the model and its 4 derivatives (~12
    flop), the residual with its compensated square sum (~6) and the normal
    equations (15 FMA): ~68 flop; ~5 for the cell coordinate, ~100 for the 4x4
    solve, ~384 for the Huber terms of the current and trial points; plus the
    evaluation at the start point amortised over the n_lm steps of a fit."""
    return round((68 * frames + 5) * (1 + 1 / n_lm) + 100 + 384)


LM_FLOPS_PER_VOXEL_STEP = lm_flops_per_voxel_step(frames=S.WORKLOADS["pr2"].n_frames)


# DRAM traffic (read + write) per launch measured by ncu on the 16-central-plane
# case of this workload and scaled by 127/16 (traffic grows with the number of
# planes: every kernel touches each plane's data independently), valid while
# the kernel's source file is unchanged (sha256 prefix); see profiles/.
TRAFFIC = {
    "lm_step": {"bytes": 473.66e6 * 127 / 16, "src": "kinetics.cu", "sha": "94e46969dddda74f"},
    "bwd_osl": {"bytes": 515.07e6 * 127 / 16, "src": "projector.cu", "sha": "9749039f5d8668f2"},
    "fwd_ratio": {"bytes": 211.53e6 * 127 / 16, "src": "projector.cu", "sha": "9749039f5d8668f2"},
    "tac_eval": {"bytes": 153.52e6 * 127 / 16, "src": "kinetics.cu", "sha": "94e46969dddda74f"},
}


def joseph_nnz_per_subset(W):
    """Mean number of nonzero Joseph-matrix entries (voxel, bin) of one plane
    and one subset: every in-grid interpolation partner with a positive weight
    of every ray sample (the positions the projector kernels compute, here in
    float64).  Each
    entry moves one M-frame vector through the SM data path: an image vector
    in the forward projection, a ratio vector in the back-projection."""
    B, A = W.n_bins, W.n_angles
    bf = np.arange(B) - 0.5 * (B - 1)
    total = 0
    for a in range(A):
        c, s = np.cos(a * np.pi / A), np.sin(a * np.pi / A)
        if A <= 4 * a <= 3 * A:                            # steps over x
            beta, gamma, n_major, n_minor = W.bin_mm / (s * W.vox_mm), -c / s, W.nx, W.ny
        else:
            beta, gamma, n_major, n_minor = W.bin_mm / (c * W.vox_mm), -s / c, W.ny, W.nx
        tf = np.arange(n_major) - 0.5 * (n_major - 1)
        fr = bf[:, None] * beta + (tf[None, :] * gamma + 0.5 * (n_minor - 1))
        j0 = np.floor(fr)
        total += np.count_nonzero((j0 >= 0) & (j0 < n_minor))                    # weight 1 - f > 0
        total += np.count_nonzero((j0 >= -1) & (j0 < n_minor - 1) & (fr > j0))   # weight f > 0
    return total / W.n_subsets


L1_BYTES_PER_CYCLE = 128   # L1 / shared-memory data path of one SM


def _traffic(kernel):
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t:
        return None
    path = os.path.join(ROOT, "paper_1803_10045_b300", "csrc", t["src"])
    with open(path, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    return round(t["bytes"] / 1e9, 4) if sha == t["sha"] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p.get("hbm_gbs", 6400.0), p.get("sm_max_mhz", 2032.0), "measured"
    except OSError:
        return 6400.0, 2032.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(reps=1, seed=0):
    """Time the FP64 oracle on a bounded sample of the PR2 workload in a fresh
    single-threaded process and extrapolate to ICM iterations per second."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = (f"import json, sys; sys.path.insert(0, {ROOT!r}); import bench; "
            f"print(json.dumps(bench._oracle_sample_inner({reps}, {seed})))")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_all_cores(max_procs=64, seed=0):
    """The same oracle sample on every host core at once: one single-threaded
    process per core (planes are independent), each timing its own sample
    after a common start instant; the ICM rate of all cores together is the
    per-core rate under that load times the number of processes."""
    n = max(1, min(max_procs, len(os.sched_getaffinity(0))))
    try:                                          # ~0.3 GB per process: stay in a quarter
        with open("/proc/meminfo") as f:          # of the available host memory
            avail_gb = next(int(l.split()[1]) for l in f if l.startswith("MemAvailable")) / 2**20
        n = max(1, min(n, int(avail_gb / 4 / 0.3)))
    except (OSError, StopIteration, ValueError):
        pass
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    start_at = time.time() + 10.0 + 0.05 * n      # after every process has set up
    code = ("import json, sys; sys.path.insert(0, {root!r}); import bench; "
            "print(json.dumps(bench._oracle_sample_inner(1, {seed}, {start})))")
    procs = [subprocess.Popen([sys.executable, "-c", code.format(root=ROOT, seed=seed + i,
                                                                  start=start_at)],
                              env=env, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                              text=True) for i in range(n)]
    vals = []
    for p in procs:
        out, _ = p.communicate()
        if p.returncode == 0:
            vals.append(json.loads(out.strip().splitlines()[-1]))
    if not vals:
        return None
    per_core = statistics.median(v["value"] for v in vals)
    return {"value": per_core * len(vals), "unit": "iter/s", "cores": len(vals),
            "kind": "oracle", "cpu": _cpu_model(), "nproc": os.cpu_count(),
            "sample": f"the 1-thread sample run concurrently in {len(vals)} processes, one "
                      f"plane each; median per-process rate {per_core:.3g} iter/s x {len(vals)}"}


def _oracle_sample_inner(reps=1, seed=0, start_at=None):
    from oracle import lm as OL
    from oracle import osl as OO
    from oracle import projector as OP
    W = S.WORKLOADS["pr2"]
    ts, te = W.frames()
    dt = te - ts
    M = W.n_frames
    og = OP.Geometry(W.nx, W.ny, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    k = 5
    x = S.random_images((1, W.ny, W.nx, M), seed=seed, lo=1.0, hi=20.0)
    counts_k = S.poisson(np.full((1, len(og.subsets[k]), W.n_bins, M), 5.0), seed)
    F = 0.9 * x
    nvox = 4096
    lm_x = x.reshape(-1, M)[:nvox].reshape(1, 64, 64, M)
    lm_maps = np.broadcast_to(np.array(S.XI0)[:, None, None, None], (4, 1, 64, 64)).copy()
    lam = np.full((1, 64, 64), 1e-2)
    t_osl, t_lm = [], []
    og.P(k)                                    # system matrix of the subset (setup)
    if start_at is not None:                   # common start of concurrent samples
        time.sleep(max(0.0, start_at - time.time()))
    for _ in range(reps):
        t0 = time.perf_counter()
        OO.osl_update(og, x, k, counts_k, 1.0, dt, F=F, beta=beta_kp_for(1.0))
        t1 = time.perf_counter()
        OL.lm_step(lm_x, lm_maps, lam, ts, te, S.FENG, BETA_H, DELTA)
        t2 = time.perf_counter()
        t_osl.append(t1 - t0)
        t_lm.append(t2 - t1)
    to, tl = min(t_osl), min(t_lm)
    V_plane = W.nx * W.ny
    t_iter = W.nz * (W.n_subsets * to + N_LM * tl * V_plane / nvox)
    return {"value": 1.0 / t_iter, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": (f"one plane: one subset OSL update ({to:.3f} s) and one MAP-LM step on "
                       f"{nvox} voxels ({tl:.3f} s), FP64 numpy, 1 thread; extrapolated to "
                       f"{W.nz} planes x ({W.n_subsets} subsets + {N_LM} LM steps over "
                       f"{V_plane} voxels) = {t_iter:.0f} s per ICM iteration")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    t0 = time.perf_counter()
    vals = [oracle_sample() for _ in range(args.steps)]
    wall = time.perf_counter() - t0
    v = statistics.median(r["value"] for r in vals)
    cb = dict(vals[0])
    cb["value"] = v
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_wall_s": round(wall, 2)},
        "cpu_baseline": cb,
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ------------------------------------------------------------------ GPU arm
def build_problem(K, torch, dev, seed=0, planes=None):
    """Synthetic PR2 study on the device: true maps -> model TACs -> projection
    -> Poisson counts (80 % trues, 20 % uniform randoms).  planes < 127 keeps
    the central planes only (for small profiler captures)."""
    import dataclasses
    W = S.WORKLOADS["pr2"]
    if planes and planes != W.nz:
        W = dataclasses.replace(W, nz=planes, total_prompts=W.total_prompts * planes / W.nz)
    ts, te = W.frames()
    g = K.Geometry(W.nx, W.ny, W.nz, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    kin = K.Kinetics(ts, te, S.FENG)
    dt = torch.tensor(te - ts, dtype=torch.float32, device=dev)
    xi_all = S.phantom_pr2(W.nx, S.WORKLOADS["pr2"].nz, seed=seed)
    z0 = (xi_all.shape[1] - W.nz) // 2
    xi = torch.from_numpy(np.ascontiguousarray(xi_all[:, z0:z0 + W.nz])).to(dev)
    del xi_all
    Ft = K.tac_eval(kin, xi)
    ybar = K.forward_project(g, Ft)
    del Ft, xi
    ybar.mul_(dt)
    trues = W.total_prompts * (1 - W.randoms_frac)
    kappa = float(trues / ybar.double().sum().item())
    n_bins_total = W.nz * W.n_angles * W.n_bins
    r = (W.total_prompts * W.randoms_frac) * dt / (dt.sum() * n_bins_total)
    ybar.mul_(kappa).add_(r)
    gen = torch.Generator(device=dev).manual_seed(seed)
    counts = torch.poisson(ybar, generator=gen)
    del ybar
    return W, g, kin, dt, kappa, counts, r.contiguous()


def run_ours(args):
    import torch

    import paper_1803_10045_b300 as K
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    W, g, kin, dt, kappa, counts, r = build_problem(K, torch, dev, seed=rank, planes=args.planes)
    M = W.n_frames
    sdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[args.storage]
    x_scale = None
    if args.counts == "u16" or args.storage != "f32":
        # measured counts are integers: uint16 holds them exactly (same results
        # bit for bit as float32 counts) at half the bytes
        assert counts.max().item() < 65536
        counts = counts.to(torch.uint16)
    if args.storage != "f32":
        x_scale = K.init_level(g, dt, kappa, counts, r)     # the start image's per-frame level
    x = K.init_image(g, dt, kappa, counts, r, dtype=sdt, x_scale=x_scale)
    params = torch.empty((4, W.nz, W.ny, W.nx), device=dev)
    params[:] = torch.tensor(S.XI0, device=dev)[:, None, None, None]
    F = torch.zeros(x.shape, device=dev)
    beta_kp = beta_kp_for(kappa)
    st = K.Study(g, kin, dt, kappa, counts, x, params, F=F, randoms=r, n_lm=N_LM,
                 beta_kp=beta_kp, beta_h=BETA_H, delta=DELTA, x_scale=x_scale)
    for _ in range(args.warmup):
        st.iterate(1)
    torch.cuda.synchronize()
    # measured FFMA rate of this GPU (the LM kernel's arithmetic roofline),
    # outside the timed region
    from paper_1803_10045_b300.peaks import measure_fma_peak
    fp32_meas = measure_fma_peak(32, target_ms=60.0)

    # ---- timed region: the kernels icm_iterate issues, with events between them
    S_ = W.n_subsets
    # ratio rows at the padded pitch the fused OSL update uses internally
    rhos = {g.n_sub(k): torch.empty(g.sino_shape(K.rho_frames(M, sdt), k), device=dev, dtype=sdt)
            for k in range(S_)}
    lm_ws = torch.empty(K.lm_workspace_size(W.nx, W.ny, W.nz), dtype=torch.uint8, device=dev)

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    def step(marks):
        for k in range(S_):
            rk = rhos[g.n_sub(k)]
            K.osl_ratio(g, k, x, dt, kappa, counts, r, out=rk, x_scale=x_scale)
            marks.append(("fwd_ratio", ev()))
            K.osl_backproject(g, k, x, dt, kappa, rk, F=F, beta=beta_kp, x_scale=x_scale)
            marks.append(("bwd_osl", ev()))
        K.map_lm_fit(kin, x, params, N_LM, BETA_H, DELTA, workspace=lm_ws, x_scale=x_scale)
        marks.append(("lm_step", ev()))
        K.tac_eval(kin, params, out=F)
        marks.append(("tac_eval", ev()))

    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    marks = [("start", ev())]
    for _ in range(args.steps):
        step(marks)
    end = marks[-1][1]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = marks[0][1].elapsed_time(end)
    if dist:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = t.item()
    per = {}
    for (_, a), (name, b) in zip(marks[:-1], marks[1:]):
        per.setdefault(name, []).append(a.elapsed_time(b))
    ok = bool(torch.isfinite(params).all().item() and torch.isfinite(x).all().item())

    # ---- end to end through the public API with host buffers
    counts_h = torch.empty(counts.shape, dtype=counts.dtype, pin_memory=True)
    counts_h.copy_(counts)
    params_h = torch.empty(params.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    e0 = ev()
    # every iteration copies its counts in and its maps out; the copies of one
    # iteration overlap the compute of its neighbours
    st.iterate_host(args.steps, counts_h, params_h)
    e1 = ev()
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    value = world * args.steps / (total_ms / 1e3)
    hbm, smax, src = _peaks()
    V = W.nx * W.ny * W.nz
    es = 4 if args.storage == "f32" else 2                 # stored image / ratio element
    cs = counts.element_size()                             # counts element
    img = V * M * es
    img32 = V * M * 4                                      # F (model TACs) stays float32
    n_sub = W.n_angles // W.n_subsets
    sino_k = W.nz * n_sub * W.n_bins * M
    alg = {  # algorithmic bytes per launch
        "fwd_ratio": img + sino_k * (cs + es),             # read x, counts_k; write rho
        "bwd_osl": sino_k * es + 2 * img + img32,          # read rho, x, F; write x
        "lm_step": img + 2 * 4 * V * 4 + 2 * V * 4 + 2 * 16 * V * 4,   # x; maps, lambda and
                                                           # normal equations in/out
        "tac_eval": 4 * V * 4 + img32,
    }
    n_launch = {"fwd_ratio": S_, "bwd_osl": S_, "lm_step": N_LM, "tac_eval": 1}
    kernels = {}
    for name, ts_ in per.items():
        launches = n_launch[name] * args.steps
        avg = sum(ts_) / launches
        kernels[name] = {"launches": launches, "avg_ms": round(avg, 4),
                         "share": round(sum(ts_) / total_ms, 4),
                         "alg_GB": round(alg[name] / 1e9, 4),
                         "alg_GBps": round(alg[name] / (avg * 1e-3) / 1e9, 1),
                         "frac_hbm": round(alg[name] / (avg * 1e-3) / 1e9 / hbm, 4),
                         "traffic_GB": _traffic(name) if args.storage == "f32" else None}
    # the projectors' own limit: the frame vectors of the Joseph matrix's
    # nonzeros through the L1 / shared-memory data path, against its byte rate
    # at the SM clock measured during the timed region
    sm_mhz = clocks.get("sm_mhz") or smax
    l1_peak = N_SM * L1_BYTES_PER_CYCLE * sm_mhz * 1e6 / 1e12
    nnz = joseph_nnz_per_subset(W) * W.nz
    for name in ("fwd_ratio", "bwd_osl"):
        l1_b = nnz * M * es
        l1_tb = l1_b / (kernels[name]["avg_ms"] * 1e-3) / 1e12
        kernels[name].update({"l1_GB": round(l1_b / 1e9, 2), "l1_TBps": round(l1_tb, 2),
                              "l1_peak_TBps": round(l1_peak, 1), "frac_l1": round(l1_tb / l1_peak, 4)})
    dom = max(kernels, key=lambda n: kernels[n]["share"])
    fp32_peak = fp32_meas["flops_per_s"] / 1e12
    fp32_src = (f"measured FFMA rate, kcs_fma_peak_launch ({fp32_meas['blocks']} blocks x 256 "
                f"threads x 16 chains, {fp32_meas['ms']} ms); unit-count figure {N_SM} SM x "
                f"{FP32_LANES_PER_SM} lanes x 2 x {smax:.0f} MHz = "
                f"{N_SM * FP32_LANES_PER_SM * 2 * smax * 1e6 / 1e12:.1f}")
    lm_tf = V * LM_FLOPS_PER_VOXEL_STEP / (kernels["lm_step"]["avg_ms"] * 1e-3) / 1e12
    kernels["lm_step"].update({"flop_per_voxel_step": LM_FLOPS_PER_VOXEL_STEP,
                               "tflops": round(lm_tf, 2), "fp32_peak_tflops": round(fp32_peak, 2),
                               "frac_fp32": round(lm_tf / fp32_peak, 4)})
    if dom == "lm_step":
        ach = lm_tf
        roof = {"bound": "alu", "kernel": dom, "achieved": round(ach, 2),
                "peak": round(fp32_peak, 1), "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                "traffic": kernels[dom]["traffic_GB"], "traffic_unit": "GB/launch",
                "peak_source": fp32_src}
    else:
        ach = kernels[dom]["alg_GBps"]
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4), "traffic": kernels[dom]["traffic_GB"],
                "traffic_unit": "GB/launch",
                "peak_source": f"{src} hbm_gbs"}
    lm_ms = kernels["lm_step"]["avg_ms"]
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if W.nz == 127 else f"{WORKLOAD} [{W.nz} central planes]",
                   "voxels": V, "frames": M, "subsets": S_, "lm_steps": N_LM,
                   "l2": f"inputs larger than L2 (image series {img / 1e9:.2f} GB, counts "
                         f"{W.nz * W.n_angles * W.n_bins * M * cs / 1e9:.2f} GB)",
                   "storage": (f"float32 image and ratio, {'uint16' if cs == 2 else 'float32'} "
                               "counts" if args.storage == "f32" else
                               f"{args.storage} image and ratio with per-frame scale, uint16 counts"),
                   "randoms": "uniform per frame", "beta_kp": beta_kp, "beta_h": BETA_H,
                   "delta": DELTA},
        "roofline": roof,
        "kernels": kernels,
        "voxel_lm_fits_per_s": round(V / (N_LM * lm_ms * 1e-3), 1),
        "voxel_lm_steps_per_s": round(V / (lm_ms * 1e-3), 1),
        "gpu_launches": args.steps * (2 * S_ + N_LM + 2),   # + the start-point normal equations
        "clocks": clocks,
        "e2e": {"value": round(world * args.steps / (e2e_ms / 1e3), 4), "unit": "iter/s",
                "h2d_bytes_per_step": counts.numel() * counts.element_size(),
                "d2h_bytes_per_step": params.numel() * 4},
        "finite": ok,
    }
    if world == 1 and not args.no_serve:
        # bounded PR5 serving leg: p50/p99 study latency under a Poisson stream
        summ, det = serve_stream(K, torch, args.serve_requests, args.mean_gap, "f32",
                                 args.budget_gb, args.max_active, args.serve_iters, args.policy)
        out["serving"] = dict({
            "studies_s": round(summ["studies_per_s"], 4), "p50_s": round(summ["p50_s"], 3),
            "p99_s": round(summ["p99_s"], 3), "completed": summ["completed"],
            "rejected": summ["rejected"], "makespan_s": round(summ["makespan_s"], 2),
            "workload": SERVE_WORKLOAD}, **det)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_sample()
        out["cpu_baseline"]["cpu"] = _cpu_model()
        out["cpu_baseline"]["all_cores"] = oracle_sample_all_cores()
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


# ------------------------------------------------------------------ serving (PR5)
SERVE_CLASSES = {   # nx, nz, bins, angles, subsets, frame schedule
    "128x32x12": (128, 32, 128, 96, 8, "pr1"),
    "256x64x16": (256, 64, 256, 188, 16, "m16"),
    "344x127x24": (344, 127, 344, 252, 21, "pr2"),
}


def _serve_template(K, torch, name, storage, seed):
    """One synthetic study of a size class: brain phantom -> model TACs ->
    projection -> Poisson counts (80 % trues, 20 % uniform randoms), at the
    count density of the full workload; counts end in pinned host memory."""
    nx, nz, nb, na, ns, sched = SERVE_CLASSES[name]
    ts, te = S.schedule(S.SCHEDULES[sched])
    fov = 344 * 2.09
    g = K.Geometry(nx, nx, nz, fov / nx, nb, na, fov / nb, ns)
    kin = K.Kinetics(ts, te, S.FENG)
    dt = torch.tensor(te - ts, dtype=torch.float32, device="cuda")
    xi = torch.from_numpy(np.ascontiguousarray(S.phantom_pr2(nx, nz, seed=seed))).cuda()
    ybar = K.forward_project(g, K.tac_eval(kin, xi))
    del xi
    ybar.mul_(dt)
    W2 = S.WORKLOADS["pr2"]
    prompts = W2.total_prompts * (nx * nx * nz) / (W2.nx * W2.nx * W2.nz)
    kappa = float(prompts * (1 - W2.randoms_frac) / ybar.double().sum().item())
    r = (prompts * W2.randoms_frac) * dt / (dt.sum() * nz * na * nb)
    ybar.mul_(kappa).add_(r)
    counts = torch.poisson(ybar, generator=torch.Generator("cuda").manual_seed(seed))
    del ybar
    if storage != "f32":
        counts = counts.to(torch.uint16)
    host = torch.empty(counts.shape, dtype=counts.dtype, pin_memory=True)
    host.copy_(counts)
    return g, kin, dt, kappa, host, r.contiguous()


def serve_stream(K, torch, requests, mean_gap, storage, budget_gb, max_active, serve_iters,
                 policy, seed=0):
    """Serve `requests` studies of the three PR5 size classes arriving as a
    Poisson stream (mean gap mean_gap s) inside an HBM budget; returns the
    summary (studies/s, arrival->done latency percentiles) and details."""
    from paper_1803_10045_b300.serving import KcsExecutor, Server, StudyRequest, summarize
    tmpl = {n: _serve_template(K, torch, n, storage, i) for i, n in enumerate(SERVE_CLASSES)}
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(mean_gap, requests))
    arrivals -= arrivals[0]
    names = list(SERVE_CLASSES)
    kinds = rng.integers(0, len(names), requests)
    reqs = []
    for rid, (t, c) in enumerate(zip(arrivals, kinds)):
        g, kin, dt, kappa, host, r = tmpl[names[c]]
        reqs.append(StudyRequest(rid, float(t), g, kin, dt, kappa, host, randoms=r,
                                 n_iter=serve_iters, n_lm=N_LM, beta_kp=beta_kp_for(kappa),
                                 beta_h=BETA_H, delta=DELTA, storage=storage))
    budget = int(budget_gb * 1e9)
    ex = KcsExecutor(budget, max_active)
    torch.cuda.synchronize()
    srv = Server(ex, budget, max_active, policy=policy)
    recs = srv.run(reqs)
    torch.cuda.synchronize()
    summ = summarize(recs)
    per = {}
    for rec, c in zip(recs, kinds):
        if rec.status == "done":
            per.setdefault(names[c], []).append(rec.latency)
    return summ, {
        "requests": requests, "mean_gap_s": mean_gap, "storage": storage,
        "budget_gb": budget_gb, "max_active": max_active, "icm_iterations": serve_iters,
        "policy": policy, "peak_arena_gb": round(srv.arena.peak / 1e9, 2),
        "class_counts": {n: int((kinds == i).sum()) for i, n in enumerate(names)},
        "latency_by_class_p50_s": {n: round(float(np.percentile(v, 50)), 3)
                                   for n, v in per.items()}}


SERVE_WORKLOAD = ("PR5: Poisson arrivals, sizes 128^2x32x12 / 256^2x64x16 / 344^2x127x24 "
                  "uniformly, ICM x 10 LM steps each")


def run_serve(args):
    """Config PR5: a stream of studies of three sizes with Poisson arrivals
    served inside an HBM budget (continuous batching at ICM-iteration
    granularity); reports studies/s and arrival->done latency percentiles."""
    import torch

    import paper_1803_10045_b300 as K
    torch.cuda.set_device(0)
    sampler = ClockSampler(0)
    sampler.start()
    summ, det = serve_stream(K, torch, args.requests, args.mean_gap, args.storage,
                             args.budget_gb, args.max_active, args.serve_iters, args.policy)
    clocks = sampler.stop()
    by_class = det.pop("latency_by_class_p50_s")
    print(json.dumps({
        "metric": "studies/s (PR5 serving)", "value": round(summ["studies_per_s"], 4),
        "unit": "studies/s", "n_gpus": 1, "higher_is_better": True,
        "p50_s": round(summ["p50_s"], 3), "p99_s": round(summ["p99_s"], 3),
        "completed": summ["completed"], "rejected": summ["rejected"],
        "makespan_s": round(summ["makespan_s"], 2), "dtype": "f32", "data": "synthetic",
        "config": dict({"workload": SERVE_WORKLOAD}, **det),
        "latency_by_class_p50_s": by_class,
        "clocks": clocks}))


# ------------------------------------------------------------------ differentiation (PR4)
def run_autograd(args):
    """Config PR4: forward y = P F(theta) and its backward (exact transpose +
    analytic kinetic Jacobian transposed) for theta [8][4][64][128][128],
    128 bins x 96 angles, 16 frames; reports passes per second."""
    import torch

    import paper_1803_10045_b300 as K
    torch.cuda.set_device(0)
    nb, nx, nz, B, A = 8, 128, 64, 128, 96
    ts, te = S.schedule(S.SCHEDULES["m16"])
    g = K.Geometry(nx, nx, nb * nz, 2.0 * 344 / nx, B, A, 2.0 * 344 / B, 1)
    kin = K.Kinetics(ts, te, S.FENG)
    gen = torch.Generator("cuda").manual_seed(0)
    base = torch.tensor(S.CLASS_XI["gm"], device="cuda")[None, :, None, None, None]
    theta = (base * (0.5 + torch.rand((nb, 4, nz, nx, nx), device="cuda", generator=gen)))
    theta.requires_grad_(True)
    w = torch.rand((nb, nz, A, B, 16), device="cuda", generator=gen)

    def step():
        theta.grad = None
        y = K.forward_model(theta, g, kin)
        (y * w).sum().backward()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd_ms, tot_ms = 0.0, 0.0
    for _ in range(args.steps):
        theta.grad = None
        e[0].record()
        y = K.forward_model(theta, g, kin)
        e[1].record()
        (y * w).sum().backward()
        e[2].record()
        torch.cuda.synchronize()
        fwd_ms += e[0].elapsed_time(e[1])
        tot_ms += e[0].elapsed_time(e[2])
    n = args.steps
    print(json.dumps({
        "metric": "forward+backward passes/s (PR4 differentiable model)",
        "value": round(1e3 * n / tot_ms, 3), "unit": "passes/s", "n_gpus": 1,
        "higher_is_better": True, "ms_forward": round(fwd_ms / n, 3),
        "ms_forward_backward": round(tot_ms / n, 3), "dtype": "f32", "data": "synthetic",
        "config": {"workload": "PR4: theta [8][4][64][128][128], TAC [8][64][128][128][16], "
                               "y [8][64][96][128][16], 128 bins x 96 angles, 16 frames",
                   "note": "the timed backward includes torch's (y * w).sum() and its gradient"}}))


# ------------------------------------------------------------------ MC bias/variance
def run_mc(args):
    """Bias and variance of the kinetic maps over many noise realisations of
    config PR1 for the three methods of Sec. IV-A (INDIRECT: OSEM then a
    post-reconstruction fit; DIRECT: ICM without the spatial prior; KCS: the
    full ICM), as a function of the number of iterations.  The realisations
    are stacked as planes of one study (planes are independent through the
    whole path), so one launch sequence reconstructs all of them; the start
    level is pooled over the realisations."""
    import torch

    import paper_1803_10045_b300 as K
    torch.cuda.set_device(0)
    W = S.WORKLOADS[args.mc_workload]
    R = args.realisations
    ts, te = W.frames()
    g = K.Geometry(W.nx, W.ny, R, W.vox_mm, W.n_bins, W.n_angles, W.bin_mm, W.n_subsets)
    kin = K.Kinetics(ts, te, S.FENG)
    dt = torch.tensor(te - ts, dtype=torch.float32, device="cuda")
    paper = args.mc_workload == "paper"
    xi1 = S.phantom_paper(W.nx) if paper else S.phantom_pr1(W.nx)    # [4][1][ny][nx]
    truth = torch.from_numpy(np.ascontiguousarray(np.repeat(xi1, R, axis=1))).float().cuda()
    ybar = K.forward_project(g, K.tac_eval(kin, truth)) * dt    # every plane the same
    for trues in [float(t) for t in args.mc_trues.split(",")]:
        for beta_kp in [float(b) for b in args.mc_beta_kp.split(",")]:
            for beta_h in [float(b) for b in args.mc_beta_h.split(",")]:
                _mc_case(args, K, torch, W, R, g, kin, dt, ybar, xi1, paper, trues, beta_kp,
                         beta_h)


def _mc_case(args, K, torch, W, R, g, kin, dt, ybar, xi1, paper, trues, beta_kp, beta_h):
    M = W.n_frames
    kappa = float(trues / ybar[0].double().sum().item())
    counts = torch.poisson(ybar * kappa, generator=torch.Generator("cuda").manual_seed(args.seed))
    checkpoints = sorted({int(c) for c in args.mc_iters.split(",")})
    lab = S.labels_paper(W.nx) if paper else S.labels_pr1(W.nx)
    classes = ({"inner": 3, "middle": 2, "outer": 1} if paper     # blood (K1 = 0) excluded
               else {"gm": 2, "wm": 3, "bg": 1})
    xi_np = xi1[:, 0]
    ki_true = xi_np[0] * xi_np[2] / np.maximum(xi_np[1] + xi_np[2], 1e-12)
    start = torch.tensor(S.XI0, dtype=torch.float32, device="cuda")

    def stats(params):
        p = params.double().cpu().numpy()                       # [4][R][ny][nx]
        ki = p[0] * p[2] / np.maximum(p[1] + p[2], 1e-12)
        out = {}
        for cname, code in classes.items():
            m = lab == code
            for pname, est, tru in (("K1", p[0], xi_np[0]), ("k3", p[2], xi_np[2]),
                                    ("Ki", ki, ki_true)):
                e = est[:, m]                                   # [R][voxels]
                t = tru[m]
                out[f"{cname}_{pname}"] = {
                    "bias_pct": round(100 * float(np.mean((e.mean(0) - t) / t)), 3),
                    "std_pct": round(100 * float(np.mean(e.std(0, ddof=1) / t)), 3)}
        return out

    result = {}
    t0 = time.perf_counter()
    for method in ("indirect", "direct", "kcs"):
        x = K.init_image(g, dt, kappa, counts)
        params = torch.empty((4, R, W.ny, W.nx), device="cuda")
        params[:] = start[:, None, None, None]
        st = K.Study(g, kin, dt, kappa, counts, x, params, n_lm=N_LM, beta_kp=beta_kp,
                     beta_h=beta_h, delta=DELTA, method=method)
        done = 0
        result[method] = {}
        for c in checkpoints:
            st.iterate(c - done)
            done = c
            if method == "indirect":
                params[:] = start[:, None, None, None]
                st.fit(N_LM)
            torch.cuda.synchronize()
            result[method][str(c)] = stats(params)
    wall = time.perf_counter() - t0
    print(json.dumps({
        "metric": f"MC bias/std of kinetic maps ({args.mc_workload})", "unit": "% of the true value",
        "realisations": R, "checkpoints": checkpoints, "seed": args.seed,
        "config": {"workload": (f"{args.mc_workload}: 64x64, {M} frames, 96 bins x 90 angles, "
                                f"4 subsets, {trues:g} trues per realisation, beta_kp "
                                f"{beta_kp:g}, beta_h {beta_h:g} (KCS), delta 0.01, 10 LM "
                                "steps per iteration"),
                   "trues": trues, "beta_kp": beta_kp, "beta_h": beta_h,
                   "wall_s": round(wall, 2)},
        "results": result}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", choices=["f32", "bf16", "f16"], default="f32")
    ap.add_argument("--counts", choices=["u16", "f32"], default="u16",
                    help="storage of the measured counts (integers: uint16 is exact)")
    ap.add_argument("--planes", type=int, default=127,
                    help="central planes of the workload (127 = full; fewer for profiler captures)")
    ap.add_argument("--serve", action="store_true",
                    help="config PR5: serve a Poisson stream of studies of three sizes")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--serve-requests", type=int, default=40,
                    help="requests of the serving leg of the default line")
    ap.add_argument("--no-serve", action="store_true",
                    help="leave the serving leg out of the default line")
    ap.add_argument("--mean-gap", type=float, default=0.5)
    ap.add_argument("--budget-gb", type=float, default=32.0)
    ap.add_argument("--max-active", type=int, default=16)
    ap.add_argument("--serve-iters", type=int, default=10)
    ap.add_argument("--policy", choices=["fifo", "backfill"], default="fifo")
    ap.add_argument("--autograd", action="store_true",
                    help="config PR4: time the differentiable forward model and its backward")
    ap.add_argument("--mc", action="store_true",
                    help="bias/variance of INDIRECT, DIRECT and KCS over PR1 noise realisations")
    ap.add_argument("--realisations", type=int, default=100)
    ap.add_argument("--mc-iters", default="1,2,5,10,20")
    ap.add_argument("--mc-workload", choices=["pr1", "paper"], default="pr1")
    ap.add_argument("--mc-trues", default="1e6", help="comma-separated expected trues per realisation")
    ap.add_argument("--mc-beta-kp", default="0.1", help="comma-separated kinetics-prior weights")
    ap.add_argument("--mc-beta-h", default="0.1", help="comma-separated Huber weights (KCS)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    if args.autograd:
        run_autograd(args)
    elif args.mc:
        run_mc(args)
    elif args.serve:
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
