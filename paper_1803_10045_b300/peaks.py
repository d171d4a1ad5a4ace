"""Measured arithmetic peaks of the current GPU (FFMA and DFMA issue rates).

The roofline of a kernel bound by float32 arithmetic needs the float32
multiply-add rate of the GPU it runs on; this module measures it (and the
float64 rate) with the library's probe kernel (kcs_fma_peak_launch: 16
independent multiply-add chains per thread, several blocks per SM), timed with
CUDA events on the current stream, rather than deriving it from unit counts
and the nominal clock.

    python -m paper_1803_10045_b300.peaks [out.json]

prints (and writes) both rates with the SM clock sampled by nvidia-smi during
the measurement.
"""
from __future__ import annotations

import ctypes as C
import json
import subprocess
import sys
import threading
import time

import torch

from ._lib import check, lib


def measure_fma_peak(precision=32, target_ms=60.0, repeats=3):
    """Best of `repeats` timed probe launches of about target_ms each on the
    current device: dict(flops_per_s, ms, blocks, iters, flops)."""
    dev = torch.cuda.current_device()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * n_sm
    sink = torch.empty(blocks, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    flops = C.c_double()

    def timed(iters):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        check(lib.kcs_fma_peak_launch(precision, blocks, iters, C.byref(flops),
                                      C.c_void_p(sink.data_ptr()), stream))
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    timed(64)                                  # load the module, warm up
    iters = 256
    ms = timed(iters)
    while ms < 5.0:                            # calibrate the loop length
        iters *= 4
        ms = timed(iters)
    iters = max(1, int(iters * target_ms / ms))
    best = min(timed(iters) for _ in range(repeats))
    return {"flops_per_s": flops.value / (best * 1e-3), "ms": round(best, 3), "blocks": blocks,
            "iters": iters, "flops": flops.value}


class _Clocks:
    """nvidia-smi SM clock samples (MHz) while a measurement runs."""

    def __init__(self, index):
        self.index, self.samples, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            try:
                self.samples.append([float(v) for v in line.split(",")])
            except ValueError:
                pass

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            self.proc.wait()

    def median(self):
        if not self.samples:
            return None, None
        sm = sorted(s[0] for s in self.samples)
        return sm[len(sm) // 2], max(s[1] for s in self.samples)


def measure_peaks(target_ms=60.0):
    """FFMA and DFMA rates (TFLOP/s) with the SM clock sampled during each."""
    out = {"gpu": torch.cuda.get_device_name(), "sms": torch.cuda.get_device_properties(
        torch.cuda.current_device()).multi_processor_count}
    for prec, name in ((32, "fp32"), (64, "fp64")):
        with _Clocks(torch.cuda.current_device()) as ck:
            r = measure_fma_peak(prec, target_ms=target_ms, repeats=5)
        mhz, max_mhz = ck.median()
        rate = r["flops_per_s"]
        out[name] = {"tflops": round(rate / 1e12, 3), "ms": r["ms"], "blocks": r["blocks"],
                     "iters": r["iters"], "sm_mhz_median": mhz, "sm_max_mhz": max_mhz,
                     "flop_per_cycle_per_sm": (round(rate / (mhz * 1e6 * out["sms"]), 2)
                                               if mhz else None)}
    out["fp64_to_fp32"] = round(out["fp64"]["tflops"] / out["fp32"]["tflops"], 5)
    out["how"] = ("kcs_fma_peak_launch: 8 blocks of 256 threads per SM, 16 independent "
                  "multiply-add chains per thread, best of 5 launches of ~60 ms timed with "
                  "CUDA events; a multiply-add counts 2 flop")
    return out


if __name__ == "__main__":
    res = measure_peaks()
    print(json.dumps(res, indent=1))
    if len(sys.argv) > 1:
        with open(sys.argv[1], "w") as f:
            json.dump(res, f, indent=1)
