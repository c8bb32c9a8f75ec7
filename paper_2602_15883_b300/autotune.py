"""Autotuner for the grouped training kernels: kernel variant, point tiles
and work schedule.

Axes, searched one after the other (coordinate search, each candidate timed
with CUDA events on whole gradient evaluations - no parameter update, so
tuning leaves the state untouched - and the fastest kept):

1. the arithmetic of the contractions, where the width offers two kernel
   families (width 128: FP32 FFMA or the tcgen05 3xTF32 kernels, which meet
   the same error bounds), when the caller asks for it (``precisions``);
2. the register tiles of the jet and value kernels of that family (the FP32
   kernels are instantiated with two each, ``dpinn_tile_options``);
3. how many tiles a work item holds, which trades load balance (many small
   items finish together) against per-item overhead (the net's small
   tensors, one gradient partial per item to reduce), for the jet and the
   value items;
4. the order in which the persistent CTAs take items (longest first, or net
   order).

The result is cached in a JSON file keyed by the architecture, the point
counts, the GPU and the library build.
"""
from __future__ import annotations

import json
import math
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "dpinn", "autotune.json")


def cache_path() -> str:
    return os.environ.get("DPINN_AUTOTUNE_CACHE", DEFAULT_CACHE)


_BUILD_IDS: dict = {}


def build_id() -> str:
    """Identity of the loaded library build: a hash of libdpinn.so's bytes, so
    that schedules tuned on other kernels are not reused while a rebuild of
    the same sources keeps its cache entries."""
    import hashlib
    from .binding import LIB_PATH
    try:
        st = os.stat(LIB_PATH)
    except OSError:
        return "nobuild"
    key = (st.st_size, st.st_mtime_ns)
    if key not in _BUILD_IDS:
        h = hashlib.sha256()
        with open(LIB_PATH, "rb") as f:
            for chunk in iter(lambda: f.read(1 << 22), b""):
                h.update(chunk)
        _BUILD_IDS[key] = h.hexdigest()[:16]
    return _BUILD_IDS[key]


def schedule_key(cfg: dict, n_res: int, n_val: int, n_nets: int, device: str, build: str = "",
                 precisions=None) -> str:
    """Architecture, precision (or the set of precisions searched),
    activation, log2 buckets of the residual / value point totals, GPU and
    library build."""
    din = cfg["d_space"] + cfg["unsteady"]
    b = lambda n: int(math.floor(math.log2(max(n, 1))))
    prec = cfg.get("precision", 0) if precisions is None else "+".join(str(int(p)) for p in sorted(precisions))
    return (f"W{cfg['width']}-L{cfg['depth']}-din{din}-ds{cfg['d_space']}-nets{n_nets}"
            f"-prec{prec}-act{cfg.get('activation', 0)}"
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


def _time_eval(handle, reps, stream):
    """Median time (ms) of `reps` gradient evaluations after one warm-up."""
    import torch
    handle.eval_grad(stream)       # warm-up after a rebuild
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
    for r in range(reps):
        ev[2 * r].record(stream)
        handle.eval_grad(stream)
        ev[2 * r + 1].record(stream)
    torch.cuda.synchronize()
    ms = sorted(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(reps))
    return ms[len(ms) // 2]


def _apply(handle, c):
    """Set a full candidate (precision, tiles, schedule) on the handle."""
    if "precision" in c and handle.get_precision() != c["precision"]:
        handle.set_precision(c["precision"])
    handle.set_tiles(c.get("jet_tile", 0), c.get("val_tile", 0))
    handle.set_schedule(c["jet_tiles"], c["val_tiles"], c["order"])


def autotune(handle, n_res: int, n_val: int, reps: int = 3, use_cache: bool = True,
             jet_candidates=(0, 2, 4, 8, 16, 32, 64), val_candidates=(0, 2, 8, 32), precisions=None,
             verbose=False):
    """Pick and set the fastest (precision, tiles, schedule) for ``handle``;
    returns it with its time and the trials.  ``precisions``: None keeps the
    handle's arithmetic; a tuple (e.g. (0, 1)) also searches it (width 128
    only offers both)."""
    import torch
    stream = torch.cuda.current_stream()
    dev = torch.cuda.get_device_name(handle.cfg.get("device", 0)).replace(" ", "_")
    if precisions is not None and handle.cfg["width"] != 128:
        precisions = None
    key = schedule_key(handle.cfg, n_res, n_val, handle.n_nets, dev, build_id(), precisions)
    if use_cache:
        hit = load_cache().get(key)
        if hit:
            _apply(handle, hit)
            return dict(hit, cached=True)
    trials = []

    def run(c):
        _apply(handle, c)
        ms = _time_eval(handle, reps, stream)
        trials.append((dict(c), ms))
        if verbose:
            print("autotune", c, f"{ms:.3f} ms")
        return ms

    best = {"precision": handle.get_precision(), "jet_tile": 0, "val_tile": 0,
            "jet_tiles": 0, "val_tiles": 0, "order": 0}
    best_ms = run(best)
    # 1. arithmetic
    for p in (precisions or ()):
        c = dict(best, precision=int(p))
        if c != best:
            ms = run(c)
            if ms < best_ms:
                best, best_ms = c, ms
    _apply(handle, best)
    # 2. register tiles of the chosen family (all combinations, at most 2 x 2)
    jo, vo = handle.tile_options()
    for j in range(len(jo)):
        for v in range(len(vo)):
            c = dict(best, jet_tile=j, val_tile=v)
            if c == best:
                continue   # the default tiles, already timed
            ms = run(c)
            if ms < best_ms:
                best, best_ms = c, ms
    # 3-4. chunk sizes of the jet and value items, then the item order
    for name, cands in (("jet_tiles", jet_candidates), ("val_tiles", val_candidates), ("order", (0, 1))):
        for cnd in cands:
            c = dict(best)
            c[name] = cnd
            if c == best:
                continue
            ms = run(c)
            if ms < best_ms:
                best, best_ms = c, ms
    _apply(handle, best)
    sched = handle.get_schedule()
    out = dict(best, ms=best_ms, trials=len(trials), tile_points=sched["tile_points"],
               precision_ms={str(c["precision"]): round(m, 4) for c, m in trials
                             if c.get("jet_tile", 0) == 0 and c.get("val_tile", 0) == 0
                             and c["jet_tiles"] == 0 and c["val_tiles"] == 0 and c["order"] == 0})
    if use_cache:
        store_cache(key, out)
    return dict(out, cached=False)
