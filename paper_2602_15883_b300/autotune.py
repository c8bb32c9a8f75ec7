"""Schedule autotuner for the grouped training kernels.

The persistent kernels take (net, point-chunk) work items from an atomic
counter.  How many tiles a chunk holds trades load balance (many small items
finish together) against per-item overhead (loading the net's small tensors,
one gradient partial per item to reduce); the order decides whether the
long items of uneven nets start first.  ``autotune`` times candidate
schedules with CUDA events on whole gradient evaluations (no parameter
update, so tuning leaves the state untouched) and keeps the fastest,
caching it in a JSON file keyed by the architecture, the point counts and
the GPU.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dpinn", "autotune.json")


def cache_path() -> str:
    return os.environ.get("DPINN_AUTOTUNE_CACHE", DEFAULT_CACHE)


def build_id() -> str:
    """Identity of the loaded library build (size and modification time of
    libdpinn.so): schedules tuned on another build are not reused."""
    from .binding import LIB_PATH
    try:
        st = os.stat(LIB_PATH)
        return f"{st.st_size}-{st.st_mtime_ns}"
    except OSError:
        return "nobuild"


def schedule_key(cfg: dict, n_res: int, n_val: int, n_nets: int, device: str, build: str = "") -> str:
    """Architecture, precision, activation, log2 buckets of the residual /
    value point totals, GPU and library build."""
    din = cfg["d_space"] + cfg["unsteady"]
    b = lambda n: int(math.floor(math.log2(max(n, 1))))
    return (f"W{cfg['width']}-L{cfg['depth']}-din{din}-ds{cfg['d_space']}-nets{n_nets}"
            f"-prec{cfg.get('precision', 0)}-act{cfg.get('activation', 0)}"
            f"-res2^{b(n_res)}-val2^{b(n_val)}-{device}-{build}")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, value: dict, path: str | None = None) -> None:
    path = path or cache_path()
    data = load_cache(path)
    data[key] = value
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_schedule(handle, sched, reps, stream):
    import torch
    handle.set_schedule(**sched)
    handle.eval_grad(stream)       # warm-up after the rebuild
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    ms = []
    for r in range(reps):
        ev[2 * r].record(stream)
        handle.eval_grad(stream)
        ev[2 * r + 1].record(stream)
    torch.cuda.synchronize()
    ms = sorted(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))
    return ms[len(ms) // 2]


def autotune(handle, n_res: int, n_val: int, reps: int = 3, use_cache: bool = True,
             jet_candidates=(0, 2, 4, 8, 16, 32, 64), val_candidates=(0, 2, 8, 32), verbose=False):
    """Pick and set the fastest schedule for ``handle``; returns it with its time."""
    import torch
    stream = torch.cuda.current_stream()
    dev = torch.cuda.get_device_name(handle.cfg.get("device", 0)).replace(" ", "_")
    key = schedule_key(handle.cfg, n_res, n_val, handle.n_nets, dev, build_id())
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            handle.set_schedule(hit["jet_tiles"], hit["val_tiles"], hit["order"])
            return dict(hit, cached=True)
    best = {"jet_tiles": 0, "val_tiles": 0, "order": 0}
    best_ms = _time_schedule(handle, best, reps, stream)
    trials = [(dict(best), best_ms)]
    # coordinate search: jet chunk, then value chunk, then item order
    for name, cands in (("jet_tiles", jet_candidates), ("val_tiles", val_candidates), ("order", (0, 1))):
        for c in cands:
            s = dict(best)
            s[name] = c
            if s == best:
                continue
            ms = _time_schedule(handle, s, reps, stream)
            trials.append((s, ms))
            if verbose:
                print("autotune", s, f"{ms:.3f} ms")
            if ms < best_ms:
                best, best_ms = s, ms
    handle.set_schedule(**best)
    out = dict(best, ms=best_ms, trials=len(trials))
    if use_cache:
        store_cache(key, out)
    return dict(out, cached=False)
