"""Benchmark: residual points per second of one full training step of all
subdomain networks (grouped jet forward + residuals + losses + reverse pass +
Adam) on synthetic analytic-flow data.

Default workload: the 3-D unsteady Beltrami flow decomposed into 4 x 4 x 2
space x 4 time = 128 nets of 6 x 128 tanh, residual points per net drawn
from a truncated power law n^-1.2 on [2,048, 65,536] (about 1.97 M in all),
2,048 noisy velocity points per net and 1,024 points per shared face (352
faces); the headline runs the FP32 kernels (the paper's arithmetic).  The
same line carries the tcgen05 3xTF32 variant of that workload (key
"tf32x3"), the 32-net Taylor-Green workload (key "tgv") and the paper's 3-D
cylinder network shape (key "cylinder3d": 8 nets of 8 x 200 sin, the
streamed-weight kernel, at most 10 timed steps) measured the same way.
--workload picks another headline configuration.

Prints one JSON line (rank 0).  `value` is device-timed with CUDA events
around each step, L2 flushed (a 512 MiB buffer is written) between steps;
`e2e` is the same metric through the C ABI with the residual points copied
from pinned host memory and the loss record copied back every step.
`roofline.traffic` is the DRAM traffic per launch of the same kernel from an
ncu capture of the same workload (profiles/ncu_traffic.json),
reported only while the kernel's sources are the captured ones;
`roofline.probe_tflops` is the FP32 FMA rate measured now by the library's
probe kernel.  `plain_form` also times the per-net loop captured in one CUDA
graph.  Other workloads: kovasznay, beltrami32, beltrami128 (width 128, the
tensor-core kernels by default), cylinder2d and cylinder3d (the paper's
cylinder network shapes).
--impl reference times the FP64 CPU oracle on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import platform
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2602_15883_b300 import synth  # noqa: E402

METRIC = "residual-points/s per train step (fwd+jets+bwd+Adam)"


def flops_per_point(cfg, jets=True):
    """Algorithmic FLOPs per point of forward + reverse (3x the forward).

    Forward with jets: 2*C*W^2*(L-1) (hidden contractions) + 2*W*(d_in + C*d_out)
    (first and output maps); value-only: the same with C = 1."""
    W, L = cfg["width"], cfg["depth"]
    din, dout = synth.d_in(cfg), synth.d_out(cfg)
    C = din + 2 if jets else 1
    return 3 * (2 * C * W * W * (L - 1) + 2 * W * (din + C * dout))


def step_flops(cfg, pb):
    n_val = int(pb.obs_counts.sum()) + 2 * int(pb.face_counts.sum())
    return flops_per_point(cfg, True) * pb.n_res + flops_per_point(cfg, False) * n_val


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.p = None
        self.rows = []
        self.window = None

    def start(self):
        """Start sampling (every 100 ms); give nvidia-smi a second to come up."""
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except OSError:
            self.p = None
            return
        import threading
        self._stamped = []

        def reader():
            for line in self.p.stdout:
                self._stamped.append((time.time(), line))
        self._t = threading.Thread(target=reader, daemon=True)
        self._t.start()
        time.sleep(1.0)

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.p is None:
            return
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self._t.join(timeout=2)
        t0, t1 = self.window or (0, 1e30)
        stamped = [(t, l) for t, l in self._stamped]
        inside = [l for t, l in stamped if t0 - 0.15 <= t <= t1 + 0.15]
        if not inside and stamped:   # region shorter than the sampling period
            mid = 0.5 * (t0 + t1)
            inside = [min(stamped, key=lambda x: abs(x[0] - mid))[1]]
        for line in inside:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append(f)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        num = lambda x: x.replace(".", "", 1).isdigit()
        sm = [float(r[1]) for r in self.rows if num(r[1])]
        mx = [float(r[2]) for r in self.rows if num(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in self.rows if num(r[3])]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz):
    # 148 SMs x 128 FP32 lanes x 2 FLOP per FFMA x clock
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


PRECISIONS = {"fp32": 0, "tf32x3": 1}


def max_over_ranks(dist, values, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest
    replica's times); ``device`` "cuda" for NCCL, "cpu" for gloo."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_value(world, n_res_per_rank, steps, total_ms_max):
    """Whole-job residual points per second: every replica's points over the
    slowest replica's time (weak scaling: each rank runs its own problem)."""
    return world * n_res_per_rank * steps / (total_ms_max / 1e3)


TRAFFIC_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "ncu_traffic.json")


def kernel_source_sha256(files):
    """SHA-256 over the named source files (paths relative to the repository
    root): the sources that define a captured kernel."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(workload, precision, scale=1):
    """DRAM bytes (read + write) per launch of the jet kernel from an ncu
    capture of this workload, or None when there is none, the sources that
    define the kernel changed since it was taken, or the run is a reduced
    (--scale) case that the capture does not describe."""
    if scale != 1:
        return None
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    for c in rec.get("captures", []):
        if c["workload"] == workload and c["precision"] == precision:
            try:
                same = c.get("sources_sha256") == kernel_source_sha256(c.get("sources", []))
            except OSError:
                return None
            return c["dram_bytes_per_launch"] if same and c.get("sources") else None
    return None


def tf32_tensor_peak_tflops(pk):
    # dense TF32 from the measured dense bf16 (cuBLAS) burst figure and the
    # nominal B300 ratio (1.1 / 2.25 PFLOP/s)
    return float(pk.get("bf16_tflops", 1800.0)) * 1.1 / 2.25


def make_problem(args, rank=0):
    cfg = synth.config(args.workload)
    pb = synth.make_problem(cfg, seed=args.seed + rank)
    return cfg, pb


def cpu_baseline(cfg, pb, budget_s=15.0):
    """The FP64 oracle on a bounded sample: every net keeps the same
    architecture, faces and structure, with 1/f of its points."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    f = 64
    while True:
        sub = synth.make_problem(cfg, seed=pb.seed,
                                 res_counts=np.maximum(pb.res_counts // f, 1),
                                 obs_counts=np.maximum(pb.obs_counts // f, 1),
                                 face_counts=np.maximum(pb.face_counts // f, 1))
        ora = oracle.Oracle(cfg, sub)
        th = np.asarray(sub.theta0, np.float64)
        t0 = time.perf_counter()
        ora.step(th, np.zeros_like(th), np.zeros_like(th), 0)
        dt = time.perf_counter() - t0
        if dt > 1.0 or f == 1:
            break
        f = max(1, f // 8)
    reps = max(1, int(budget_s / max(dt, 1e-3)))
    reps = min(reps, 20)
    t0 = time.perf_counter()
    for _ in range(reps):
        ora.step(th, np.zeros_like(th), np.zeros_like(th), 0)
    dt = (time.perf_counter() - t0) / reps
    return {"value": sub.n_res / dt, "unit": "residual-points/s", "cores": cores, "cpu": cpu_model(), "kind": "oracle",
            "sample": f"all {synth.n_nets(cfg)} nets with 1/{f} of their points ({sub.n_res} residual pts), "
                      f"FP64 loss+gradient+Adam, {reps} steps"}


def cpu_model():
    """The host CPU's model name (read at run time), for the CPU baseline."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, pb = make_problem(args)
    cb = cpu_baseline(cfg, pb, budget_s=max(5.0, 2.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "residual-points/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "n_nets": synth.n_nets(cfg), "residual_points": pb.n_res},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "residual-points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def plain_form_rate(cfg, pb, steps=2):
    """Plain form (per-net eager PyTorch autograd loop, FP32) on the GPU."""
    import torch
    from baseline.plain_form import PlainForm
    pf = PlainForm(pb, device="cuda", dtype=torch.float32)
    pf.step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        pf.step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    out = {"value": pb.n_res / dt, "unit": "residual-points/s", "ms_per_step": dt * 1e3,
           "kind": "per-net eager PyTorch autograd double backward + torch.optim.Adam, FP32"}
    # the same step captured in one CUDA graph (as the paper's pipeline replays its step)
    try:
        del pf
        torch.cuda.empty_cache()
        pg = PlainForm(pb, device="cuda", dtype=torch.float32).capture()
        pg.replay()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(max(steps, 5)):
            pg.replay()
        torch.cuda.synchronize()
        dg = (time.perf_counter() - t0) / max(steps, 5)
        out["graph_captured"] = {"value": pb.n_res / dg, "ms_per_step": dg * 1e3,
                                 "kind": "the same step captured in one CUDA graph (capturable Adam), FP32"}
    except Exception as ex:   # context only: record why it could not run
        out["graph_captured"] = {"error": str(ex)[:200]}
    return out


def serving_leg(seconds=5.0, rate=200.0, train_steps=20, seed=0, precision="tf32x3"):
    """Continuous-batching serving of the trained 32-net Beltrami ensemble:
    Poisson arrivals, log-uniform 1k-1M point clouds, 10 % with residuals,
    8 GB in-flight memory cap; p50/p99 latency and points/s.  The ensemble
    (width 128) trains and answers on the tensor-core kernels by default."""
    from paper_2602_15883_b300.binding import Dpinn
    from paper_2602_15883_b300.serve import Server, latency_summary, poisson_load
    cfg = synth.config("beltrami32", precision=PRECISIONS[precision])
    pb = synth.make_problem(cfg, seed=seed)
    d = Dpinn(cfg)
    d.set_problem(pb)
    d.step(train_steps)
    d.loss()
    srv = Server(d, slots=4, mem_cap_bytes=8 << 30, max_batch_points=1 << 21).start()
    try:
        # warm-up: every slot serves small and large requests, values and
        # residuals (first launches load their kernels), then a light load
        warm = [srv.submit(synth.query_points(cfg, n, seed=seed + 10 + i), res)
                for i, (n, res) in enumerate([(n, res) for res in (False, True) for n in (1000, 1 << 20)] * 4)]
        for r in warm:
            r.done.wait()
        del warm, r
        poisson_load(srv, cfg, rate_hz=20.0, duration_s=0.5, seed=seed + 1)
        half = poisson_load(srv, cfg, rate_hz=rate / 2, duration_s=seconds, seed=seed + 3, client_buffers=True)
        reqs = poisson_load(srv, cfg, rate_hz=rate, duration_s=seconds, seed=seed + 2, client_buffers=True)
    finally:
        srv.stop()
    out = latency_summary(reqs)
    out.update({"workload": "beltrami32 ensemble (32 nets of 8x128) after %d training steps" % train_steps,
                "arrivals": f"Poisson {rate:g} req/s for {seconds:g} s", "points_per_request": "log-uniform 1e3..1e6",
                "residual_fraction": 0.1, "mem_cap_gb": 8, "slots": 4, "precision": precision,
                "slot_points": srv.max_points, "device_bytes": srv.device_bytes,
                "max_concurrent_batches": srv.max_concurrent,
                "offered_points_per_s": sum(r.n for r in reqs) / seconds})
    h = latency_summary(half)
    h.update({"arrivals": f"Poisson {rate / 2:g} req/s for {seconds:g} s",
              "offered_points_per_s": sum(r.n for r in half) / seconds})
    out["at_half_load"] = h
    d.close()
    return out


def measure(args, workload, precision, rank, world, local, dist, stream, clocks=True):
    """Device-timed training steps, per-kernel times, roofline and the
    end-to-end rate of one (workload, precision) on this rank's replica.
    Returns the handle's problem and a dict of results."""
    import torch
    from paper_2602_15883_b300.binding import POINTS_RESIDUAL, Dpinn
    cfg = synth.config(workload)
    pb = synth.make_problem(cfg, seed=args.seed + rank)
    if args.scale > 1:   # profiling captures only: every point set divided by the factor
        base = pb
        pb = synth.make_problem(cfg, seed=args.seed + rank, res_counts=np.maximum(base.res_counts // args.scale, 1),
                                obs_counts=np.maximum(base.obs_counts // args.scale, 1),
                                face_counts=np.maximum(base.face_counts // args.scale, 1))
    cfg["device"] = local
    auto = precision == "auto"   # the autotuner picks the arithmetic (width 128: FP32 or 3xTF32)
    if auto and cfg["width"] != 128:
        precision, auto = "fp32", False
    cfg["precision"] = 0 if auto else PRECISIONS[precision]
    d = Dpinn(cfg)
    d.set_problem(pb)
    schedule = {"jet_tiles": 0, "val_tiles": 0, "order": 0, "tuned": False}
    if not args.no_autotune:
        from paper_2602_15883_b300 import autotune
        n_val = int(pb.obs_counts.sum() + 2 * pb.face_counts.sum())
        res = autotune.autotune(d, pb.n_res, n_val, reps=3, precisions=(0, 1) if auto else None)
        schedule = {k: res.get(k, 0) for k in ("jet_tiles", "val_tiles", "order", "jet_tile", "val_tile")}
        schedule.update(tuned=True, cached=res.get("cached", False), trials=res.get("trials"),
                        jet_tile_options=d.tile_options()[0], val_tile_options=d.tile_options()[1])
        if auto:
            schedule["variant_ms"] = {("tf32x3" if k == "1" else "fp32"): v
                                      for k, v in res.get("precision_ms", {}).items()}
    elif auto:
        d.set_precision(1)
    if args.no_autotune and args.tiles and not auto:
        d.set_tiles(*[int(x) for x in args.tiles.split(",")])
    precision = "tf32x3" if d.get_precision() == 1 else "fp32"
    cfg["precision"] = PRECISIONS[precision]
    schedule["variant"] = precision + (" (autotuned)" if auto and not args.no_autotune else "")
    schedule["tile_points"] = d.get_schedule()["tile_points"]
    schedule["jet_tile"], schedule["val_tile"] = d.get_tiles()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    d.step(args.warmup, stream)
    d.loss()
    # ---- device-timed region
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clk = Clocks(local)
    if clocks:
        clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.time()
    for i in range(args.steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        d.step(1, stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    clk.mark(w0, time.time())
    if dist:
        dist.barrier()
    ms = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    loss = d.loss()
    assert np.all(np.isfinite(loss)), "non-finite loss"
    total_ms = float(ms.sum())
    step_ms = total_ms / args.steps   # the mean, so that value = points / step time
    if dist:
        total_ms, step_ms = max_over_ranks(dist, [total_ms, step_ms], "cuda")
    value = whole_job_value(world, pb.n_res, args.steps, total_ms)

    # ---- per-kernel timing of the same kernels (events on this stream)
    kt = {}
    for i in range(max(3, min(args.steps, 10))):
        flush.fill_(0.0)
        for k, v in d.step_timed(stream).items():
            kt.setdefault(k, []).append(v)
    kms = {k: float(np.mean(v)) for k, v in kt.items()}
    jet_ms = kms.get("train_jet", float("nan"))
    if clocks:
        clk.stop()
    pk, pk_kind = peaks()
    sm_mhz = float(pk.get("sm_max_mhz", 2032.0))
    jet_flops = flops_per_point(cfg, True) * pb.n_res
    achieved = jet_flops / (jet_ms / 1e3) / 1e12
    if precision == "fp32":
        peak = fp32_alu_peak_tflops(sm_mhz)
        # context: the attainable FP32 FMA rate measured now by the library's
        # packed-FMA chain probe (a ~20 ms burst)
        from paper_2602_15883_b300.binding import probe_fp32
        cal_ms, _ = probe_fp32(2000)
        p_ms, p_flop = probe_fp32(max(1, int(2000 * 20.0 / max(cal_ms, 1e-3))))
        probe_tflops = p_flop / (p_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "probe_tflops": probe_tflops, "frac_of_probe": achieved / probe_tflops,
                    "frac": achieved / peak, "traffic": captured_traffic(workload, "fp32", args.scale),
                    "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                    "kernel": "k_pinn train (jets)" if cfg["width"] in (32, 64, 128) else "k_pinn_w train (jets)",
                    "work_per_launch": f"{flops_per_point(cfg, True)} FLOP per residual point x {pb.n_res} points",
                    "peak_source": f"148 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (max SM clock, {pk_kind})",
                    "kernel_ms": kms}
    else:
        peak = tf32_tensor_peak_tflops(pk)
        hidden = 3 * 2 * (synth.d_in(cfg) + 2) * cfg["width"] ** 2 * (cfg["depth"] - 1) * pb.n_res
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": captured_traffic(workload, "tf32x3", args.scale),
                    "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                    "kernel": "k_pinn_tc train (jets, tcgen05 3xTF32)",
                    "work_per_launch": f"{flops_per_point(cfg, True)} FLOP per residual point x {pb.n_res} points",
                    "peak_source": f"dense TF32 = measured bf16 burst x 1.1/2.25 (nominal ratio, {pk_kind})",
                    "hw_tflops_3x": 3 * hidden / (jet_ms / 1e3) / 1e12,
                    "frac_3x": 3 * hidden / (jet_ms / 1e3) / 1e12 / peak,
                    "note": "achieved counts every product once; the tensor cores execute three per product",
                    "kernel_ms": kms}

    # ---- end to end through the C ABI with host buffers: every step's points
    # are copied from pinned host memory (two buffers, alternating) and its
    # loss record copied back into pinned memory and read on the host.  The
    # loop keeps one step queued ahead: the upload of step i + 1 overlaps
    # step i, and the host reads step i's losses while step i + 1 runs.
    pinned = [torch.from_numpy(np.ascontiguousarray(pb.res_pts, np.float32)).pin_memory() for _ in range(2)]
    counts = pb.res_counts
    lbuf = [torch.zeros((d.n_nets, 6), dtype=torch.float32).pin_memory() for _ in range(2)]
    lev = [torch.cuda.Event() for _ in range(2)]
    out = np.zeros((d.n_nets, 6), np.float32)
    losses_read = 0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    d.set_points_async(POINTS_RESIDUAL, pinned[0], counts)
    for i in range(e2e_steps + 1):
        if i < e2e_steps:
            d.step(1, stream)
            d.loss_async(lbuf[i % 2], stream)
            lev[i % 2].record(stream)
            if i + 1 < e2e_steps:
                d.set_points_async(POINTS_RESIDUAL, pinned[(i + 1) % 2], counts)
        if i > 0:   # the losses of step i - 1
            lev[(i - 1) % 2].synchronize()
            out = lbuf[(i - 1) % 2].numpy().copy()
            losses_read += 1
            if not np.all(np.isfinite(out)):
                raise FloatingPointError(f"non-finite loss at end-to-end step {i - 1}")
    torch.cuda.synchronize()
    assert losses_read == e2e_steps
    e2e_s = time.perf_counter() - t0
    if dist:
        (e2e_s,) = max_over_ranks(dist, [e2e_s], "cuda")
    e2e = {"value": world * pb.n_res * e2e_steps / e2e_s, "unit": "residual-points/s",
           "h2d_bytes_per_step": int(pinned[0].numel() * 4), "d2h_bytes_per_step": int(out.nbytes)}
    r = {"value": value, "ms_per_step": step_ms, "steps": args.steps,
         "dtype": "f32" if precision == "fp32" else "tf32x3",
         "config": {"workload": workload, "n_nets": d.n_nets, "width": cfg["width"], "depth": cfg["depth"],
                    "residual_points": pb.n_res, "precision": precision,
                    "obs_points": int(pb.obs_counts.sum()), "face_points": int(pb.face_counts.sum()),
                    "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                    "l2": "flushed between steps (512 MiB write)", "schedule": schedule,
                    **({"scale": f"1/{args.scale} of every point set (profiling capture, not a bench value)"}
                       if args.scale > 1 else {})},
         "roofline": roofline, "e2e": e2e, "gpu_launches": d.launches_per_step * args.steps,
         "step_gflop": step_flops(cfg, pb) / 1e9}
    if clocks:
        r["clocks"] = clk.summary()
    d.close()
    del flush, pinned
    torch.cuda.empty_cache()
    return cfg, pb, r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="beltrami128", choices=list(synth.CONFIGS))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-baselines", action="store_true", help="skip the plain-form and CPU legs")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra measurements (the TF32x3 variant at width 128, the TGV workload)")
    ap.add_argument("--serving-seconds", type=float, default=5.0)
    ap.add_argument("--tiles", default="",
                    help="with --no-autotune: register tiles 'jet,val' as indices into the tile options")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide every point set by this factor (reduced cases for profiling captures only)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule")
    ap.add_argument("--precision", default="fp32", choices=["auto", "fp32", "tf32x3"],
                    help="hidden-layer contractions of the headline's jet kernel: FP32 FMA (the paper's "
                         "arithmetic, default), or tcgen05 3xTF32 (width 128); auto = tf32x3 where the width "
                         "allows it")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2602_15883_b300 import build
    build.build()

    width = synth.config(args.workload)["width"]
    if args.precision == "auto":
        args.precision = "tf32x3" if width == 128 else "fp32"
    stream = torch.cuda.current_stream()
    cfg, pb, head = measure(args, args.workload, args.precision, rank, world, local, dist, stream)
    extras = {}
    if not args.no_extras:
        # the other arithmetic of the width-128 kernels, and the 32-net TGV workload
        if width == 128:
            # the autotuner's choice between the two kernel families (3xTF32
            # measured faster); reported under the variant it picked
            r = measure(args, args.workload, "auto", rank, world, local, dist, stream, clocks=False)[2]
            key = "tf32x3" if r["dtype"] == "tf32x3" else "autotuned_f32"
            if key != head["dtype"]:
                extras[key] = r
        if args.workload != "tgv":
            extras["tgv"] = measure(args, "tgv", "fp32", rank, world, local, dist, stream, clocks=False)[2]
        if args.workload != "cylinder3d":
            # the paper's own 3-D network shape; a step takes about 0.2 s
            a3 = argparse.Namespace(**vars(args))
            a3.steps = min(args.steps, 10)
            extras["cylinder3d"] = measure(a3, "cylinder3d", "fp32", rank, world, local, dist, stream,
                                           clocks=False)[2]

    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": "residual-points/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": head["dtype"],
                "data": "synthetic", "config": head["config"], "roofline": head["roofline"],
                "clocks": head["clocks"], "e2e": head["e2e"], "gpu_launches": head["gpu_launches"],
                "step_gflop": head["step_gflop"]}
        line.update(extras)
        if not args.no_baselines:
            try:
                line["plain_form"] = plain_form_rate(cfg, pb)
            except Exception as ex:   # reported, not fatal
                line["plain_form"] = {"error": str(ex)[:200]}
            line["cpu_baseline"] = cpu_baseline(cfg, pb)
        if not args.no_serving and world == 1:
            try:
                line["serving"] = serving_leg(seconds=args.serving_seconds)
            except Exception as ex:   # reported, not fatal
                line["serving"] = {"error": str(ex)[:300]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()


if __name__ == "__main__":
    main()
