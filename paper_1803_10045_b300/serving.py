"""Serving many dynamic studies on one GPU with continuous batching.

Requests (one dynamic PET study each) arrive over time.  The host loop
  * admits queued studies first-come first-served while their device
    footprint fits a fixed HBM budget and an execution slot is free; the
    budget is one device allocation carved by a first-fit arena, so
    admission is an allocation that either fits or waits;
  * gives every admitted study its slot's CUDA stream and issues its ICM
    iterations (Sec. II-D) one at a time, round-robin over the active
    studies, so studies of very different sizes interleave at iteration
    granularity and run concurrently on the device;
  * polls a per-study event, and on the last iteration copies the kinetic
    maps to pinned host memory, records arrival -> done latency and returns
    the study's memory to the arena.
A request larger than the whole budget is rejected; a request can be
cancelled while queued or between two of its iterations.

The scheduling logic is independent of the device: ``Server`` drives an
executor object (``KcsExecutor`` on the GPU; tests also drive a fake one on
the CPU).  Every kernel a study runs is libkcs.so's, issued through the
package's bindings.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable

ALIGN = 256


def _up(n, a=ALIGN):
    return (int(n) + a - 1) // a * a


class Arena:
    """First-fit allocator of byte ranges inside one fixed-size region, with
    coalescing of adjacent free ranges.  Offsets are multiples of ALIGN."""

    def __init__(self, nbytes):
        self.size = int(nbytes) // ALIGN * ALIGN
        self.free_list = [(0, self.size)]       # sorted, disjoint, non-adjacent
        self.live = {}                          # offset -> length
        self.peak = 0

    @property
    def used(self):
        return sum(self.live.values())

    def alloc(self, nbytes):
        n = _up(max(int(nbytes), 1))
        for i, (off, ln) in enumerate(self.free_list):
            if ln >= n:
                if ln == n:
                    del self.free_list[i]
                else:
                    self.free_list[i] = (off + n, ln - n)
                self.live[off] = n
                self.peak = max(self.peak, self.used)
                return off
        return None

    def free(self, off):
        n = self.live.pop(off)
        fl = self.free_list
        i = 0
        while i < len(fl) and fl[i][0] < off:
            i += 1
        fl.insert(i, (off, n))
        if i + 1 < len(fl) and fl[i][0] + fl[i][1] == fl[i + 1][0]:      # merge right
            fl[i] = (fl[i][0], fl[i][1] + fl[i + 1][1])
            del fl[i + 1]
        if i > 0 and fl[i - 1][0] + fl[i - 1][1] == fl[i][0]:            # merge left
            fl[i - 1] = (fl[i - 1][0], fl[i - 1][1] + fl[i][1])
            del fl[i]


@dataclasses.dataclass
class Record:
    rid: int
    arrival: float
    footprint: int
    status: str = "queued"          # queued | active | done | rejected | cancelled
    admitted: float | None = None
    done: float | None = None
    iterations: int = 0
    result: Any = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


class Server:
    """Continuous-batching loop over an executor.

    executor.footprint(req) -> bytes; executor.admit(req, offset, slot) -> job
    (allocates the study inside the arena at offset and issues its upload and
    start image on the slot's stream); executor.issue(job) issues one ICM
    iteration; executor.ready(job) is True when everything issued so far has
    finished; executor.finish(job) issues the result copy and returns a handle
    whose readiness is polled with executor.ready; executor.result(job) returns
    the host result; executor.release(job) drops the study.
    """

    def __init__(self, executor, budget_bytes, max_active=8, clock: Callable[[], float] = None,
                 idle_sleep=50e-6, policy="fifo", max_bypass=64):
        """policy "fifo": strict first come first served (a study that does not
        fit blocks those behind it).  policy "backfill": when the oldest study
        does not fit, later ones that fit are admitted, each bypass of the
        oldest counted; once it has been bypassed max_bypass times nothing else
        is admitted before it (no starvation)."""
        if policy not in ("fifo", "backfill"):
            raise ValueError(policy)
        self.ex = executor
        self.arena = Arena(budget_bytes)
        self.policy = policy
        self.max_bypass = int(max_bypass)
        self.max_active = int(max_active)
        self.clock = clock or time.perf_counter
        self.idle_sleep = idle_sleep
        self._cancel = set()

    def cancel(self, rid):
        """Cancel request rid (queued: dropped; active: stopped after its
        iteration in flight)."""
        self._cancel.add(rid)

    def run(self, requests, on_tick: Callable[["Server", float], None] = None):
        reqs = sorted(requests, key=lambda r: r.arrival)
        recs = {r.rid: Record(r.rid, r.arrival, self.ex.footprint(r)) for r in reqs}
        queue = collections.deque()
        active = []                         # [req, job, offset, slot, phase]
        free_slots = list(range(self.max_active))[::-1]
        bypassed = {}                       # rid -> times a later study was admitted first
        t0 = self.clock()
        i = 0
        while i < len(reqs) or queue or active:
            now = self.clock() - t0
            if on_tick:
                on_tick(self, now)
            while i < len(reqs) and reqs[i].arrival <= now:
                queue.append(reqs[i])
                i += 1
            # cancellation of queued requests
            if self._cancel and queue:
                keep = collections.deque()
                for r in queue:
                    if r.rid in self._cancel:
                        recs[r.rid].status = "cancelled"
                        recs[r.rid].done = now
                    else:
                        keep.append(r)
                queue = keep
            # admission while the budget and a slot allow
            k = 0
            while k < len(queue) and free_slots:
                r = queue[k]
                rec = recs[r.rid]
                if rec.footprint > self.arena.size:
                    del queue[k]
                    rec.status, rec.done = "rejected", now
                    continue
                if k > 0 and bypassed.get(queue[0].rid, 0) >= self.max_bypass:
                    break                   # the oldest study has waited long enough
                off = self.arena.alloc(rec.footprint)
                if off is None:
                    if self.policy == "fifo":
                        break
                    k += 1                  # backfill: try a later, smaller study
                    continue
                del queue[k]
                if k > 0:
                    bypassed[queue[0].rid] = bypassed.get(queue[0].rid, 0) + 1
                slot = free_slots.pop()
                job = self.ex.admit(r, off, slot)
                rec.status, rec.admitted = "active", now
                active.append([r, job, off, slot, "run"])
            # issue: one iteration in flight per study, round-robin
            progressed = False
            still = []
            for entry in active:
                r, job, off, slot, phase = entry
                rec = recs[r.rid]
                if not self.ex.ready(job):
                    still.append(entry)
                    continue
                progressed = True
                if phase == "run" and r.rid in self._cancel:
                    rec.status, rec.done = "cancelled", self.clock() - t0
                    self.ex.release(job)
                    self.arena.free(off)
                    free_slots.append(slot)
                    continue
                if phase == "run" and rec.iterations < r.n_iter:
                    self.ex.issue(job)
                    rec.iterations += 1
                    still.append(entry)
                elif phase == "run":
                    self.ex.finish(job)
                    entry[4] = "copy"
                    still.append(entry)
                else:                       # result copy finished
                    rec.result = self.ex.result(job)
                    rec.status, rec.done = "done", self.clock() - t0
                    self.ex.release(job)
                    self.arena.free(off)
                    free_slots.append(slot)
            active = still
            if not progressed:
                if not active and not queue and i < len(reqs):
                    wait = reqs[i].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                elif self.idle_sleep:
                    time.sleep(self.idle_sleep)
        return [recs[r.rid] for r in reqs]


def summarize(records):
    """studies/s over the makespan and latency percentiles of finished studies."""
    import numpy as np
    done = [r for r in records if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(0)
    span = (max(r.done for r in done) - min(r.arrival for r in records)) if done else 0.0
    return {
        "completed": len(done),
        "rejected": sum(r.status == "rejected" for r in records),
        "cancelled": sum(r.status == "cancelled" for r in records),
        "studies_per_s": len(done) / span if span > 0 else None,
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "makespan_s": span,
    }


# ---------------------------------------------------------------- GPU executor
@dataclasses.dataclass
class StudyRequest:
    """One dynamic study: scanner geometry and frame schedule (shared, read
    only), its measured counts in pinned host memory and the ICM settings."""
    rid: int
    arrival: float
    geom: Any                      # Geometry
    kin: Any                       # Kinetics
    frame_dt: Any                  # device float32 [M]
    kappa: float
    counts_host: Any               # pinned host [Z][A][B][M], float32 or uint16
    randoms: Any = None            # device float32 [M] (per-frame uniform) or None
    n_iter: int = 10
    n_lm: int = 10
    beta_kp: float = 0.1
    beta_h: float = 0.1
    delta: float = 0.01
    storage: str = "f32"           # image / ratio storage: f32 | bf16 | f16
    start_params: tuple = (0.05, 0.10, 0.03, 0.03)


def study_layout(r):
    """Byte ranges of one study's device buffers inside its arena block, and
    the block size (the study's footprint)."""
    from ._lib import lib
    g, M = r.geom, r.kin.M
    V = g.nz * g.ny * g.nx
    es = 4 if r.storage == "f32" else 2
    parts = [
        ("counts", g.nz * g.n_angles * g.n_bins * M * r.counts_host.element_size()),
        ("x", V * M * es),
        ("F", V * M * 4),
        ("params", 4 * V * 4),
        ("scale", M * 4),
        ("ws", lib.kcs_study_workspace_size(g.handle, M)),
    ]
    out, off = {}, 0
    for name, n in parts:
        out[name] = (off, n)
        off = _up(off + n)
    return out, off


class KcsExecutor:
    """Runs studies with libkcs.so inside one device region of budget bytes."""

    def __init__(self, budget_bytes, max_active=8, device="cuda"):
        import torch
        from . import api
        self.torch, self.api = torch, api
        self.device = torch.device(device)
        self.region = torch.empty(int(budget_bytes) // ALIGN * ALIGN, dtype=torch.uint8,
                                  device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(max_active)]
        self.dtypes = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}

    def _layout(self, r):
        return study_layout(r)

    def footprint(self, r):
        return study_layout(r)[1]

    def _view(self, base, off, n, dtype, shape):
        t = self.region[base + off: base + off + n].view(dtype)
        return t.view(shape)

    def admit(self, r, base, slot):
        torch, api = self.torch, self.api
        lay, _ = self._layout(r)
        g, M = r.geom, r.kin.M
        s = self.streams[slot]
        job = {"req": r, "stream": s}
        with torch.cuda.stream(s):
            counts = self._view(base, *lay["counts"], r.counts_host.dtype, r.counts_host.shape)
            counts.copy_(r.counts_host, non_blocking=True)
            x = self._view(base, *lay["x"], self.dtypes[r.storage], g.image_shape(M))
            F = self._view(base, *lay["F"], torch.float32, g.image_shape(M))
            params = self._view(base, *lay["params"], torch.float32, (4, g.nz, g.ny, g.nx))
            ws = self._view(base, *lay["ws"], torch.uint8, (lay["ws"][1],))
            scale = None
            if r.storage != "f32":
                scale = self._view(base, *lay["scale"], torch.float32, (M,))
                api.init_level(g, r.frame_dt, r.kappa, counts, r.randoms, workspace=ws, out=scale)
            api.init_image(g, r.frame_dt, r.kappa, counts, r.randoms, out=x, workspace=ws,
                           x_scale=scale)
            for q in range(4):
                params[q].fill_(float(r.start_params[q]))
            job["study"] = api.Study(g, r.kin, r.frame_dt, r.kappa, counts, x, params, F=F,
                                     randoms=r.randoms, n_lm=r.n_lm, beta_kp=r.beta_kp,
                                     beta_h=r.beta_h, delta=r.delta, workspace=ws,
                                     x_scale=scale)
            job["params"] = params
            job["event"] = torch.cuda.Event()
            job["event"].record(s)
        return job

    def issue(self, job):
        with self.torch.cuda.stream(job["stream"]):
            job["study"].iterate(1)
            job["event"].record(job["stream"])

    def ready(self, job):
        return job["event"].query()

    def finish(self, job):
        torch = self.torch
        with torch.cuda.stream(job["stream"]):
            p = job["params"]
            job["host"] = torch.empty(p.shape, dtype=p.dtype, pin_memory=True)
            job["host"].copy_(p, non_blocking=True)
            job["event"].record(job["stream"])

    def result(self, job):
        return job["host"]

    def release(self, job):
        st = job.pop("study", None)
        if st is not None:
            st.close()
        job.clear()
