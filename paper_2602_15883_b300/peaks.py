"""Attainable FP32 FMA and TF32 tensor throughput of the GPU, measured.

    python -m paper_2602_15883_b300.peaks [--sustained-s 3]

FP32: the library's packed-FMA chain probe (dpinn_probe_fp32), as a burst
(a ~20 ms launch, median of 5) and sustained (one launch of about
--sustained-s seconds, under the power cap).  TF32: cuBLAS through
torch.matmul with TF32 enabled on 16384^3 FP32 products, burst (median of
10) and sustained (back-to-back for about --sustained-s seconds).  Prints one
JSON line; SM clocks are sampled with nvidia-smi during each measurement.
These are context for the roofline denominators that bench.py uses (FP32:
unit counts x maximum SM clock; TF32: measured bf16 x the nominal ratio).
"""
import argparse
import json
import subprocess
import time

import numpy as np

from paper_2602_15883_b300 import binding


class _Clocks:
    def __init__(self):
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=clocks.sm,power.draw", "--format=csv,noheader,nounits",
                                       "-i", "0", "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.rows = []
        if self.p is None:
            return
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        for ln in out.splitlines():
            try:
                mhz, w = (float(x) for x in ln.split(","))
                self.rows.append((mhz, w))
            except ValueError:
                pass

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "power_w_max": None}
        return {"sm_mhz": float(np.median([r[0] for r in self.rows])), "power_w_max": max(r[1] for r in self.rows)}


def fp32_probe(sustained_s):
    ms, flop = binding.probe_fp32(2000)                       # calibration launch
    per_iter_ms = ms / 2000
    it_burst = max(1, int(20.0 / per_iter_ms))
    with _Clocks() as ck:
        runs = [binding.probe_fp32(it_burst) for _ in range(5)]
    burst = float(np.median([f / (m * 1e-3) / 1e12 for m, f in runs]))
    c_burst = ck.summary()
    with _Clocks() as ck:
        m, f = binding.probe_fp32(max(1, int(sustained_s * 1e3 / per_iter_ms)))
    return {"burst_tflops": burst, "burst_clocks": c_burst,
            "sustained_tflops": f / (m * 1e-3) / 1e12, "sustained_s": m * 1e-3, "sustained_clocks": ck.summary()}


def tf32_matmul(sustained_s, n=16384):
    import torch
    torch.backends.cuda.matmul.allow_tf32 = True
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    c = torch.empty(n, n, device="cuda")
    flop = 2.0 * n ** 3
    for _ in range(3):
        torch.matmul(a, b, out=c)
    torch.cuda.synchronize()
    times = []
    with _Clocks() as ck:
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
    burst = flop / (float(np.median(times)) * 1e-3) / 1e12
    c_burst = ck.summary()
    reps = max(1, int(sustained_s * 1e3 / float(np.median(times))))
    with _Clocks() as ck:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    return {"burst_tflops": burst, "burst_clocks": c_burst, "sustained_tflops": reps * flop / (ms * 1e-3) / 1e12,
            "sustained_s": ms * 1e-3, "sustained_clocks": ck.summary(), "n": n}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sustained-s", type=float, default=3.0)
    args = ap.parse_args()
    out = {"fp32_fma_probe": fp32_probe(args.sustained_s)}
    time.sleep(1.0)
    out["tf32_cublas"] = tf32_matmul(args.sustained_s)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
