"""Continuous-batching query server for a resident ensemble.

Requests (point clouds of any size, asking for (u, v, [w], p) and optionally
the Navier-Stokes residuals) arrive at any time.  A dispatcher thread keeps
``slots`` batches in flight, each with its own query contexts, pre-allocated
buffers and two CUDA streams.  All device memory the server holds - every
slot's point, value and residual buffers and the routing scratch of its two
query contexts - is sized at start-up from the memory cap, so the server
never holds more than the cap whatever the load; a request larger than a
slot is split into slot-sized chunks that complete together as one request.
Whenever a slot is free it admits the oldest waiting requests (or chunks)
that fit the slot and the in-flight memory budget, copies
their points into one pinned staging buffer, and issues one host-to-device
copy, the value launch (requests without residual) with its device-to-host
copy on a high-priority stream, and the residual launch (jets, several times
the work per point) with its copy on a low-priority stream.  The query
kernels run one CTA per work item, so the block scheduler serves the
high-priority value work between the CTAs of a large residual request, and
value requests complete on their own event without waiting for the
residuals of their batch.  Requests that arrive while other batches run are
admitted as slots and memory free up, so the copies and kernels of
different batches overlap on the device.  Each point is computed by the same
kernel code whatever batch it lands in (no cross-point reduction), so a
request's result does not depend on the mix.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

ERR_INVALID_ARG = -1   # include/dpinn.h: DPINN_ERR_INVALID_ARG (an outside point)


@dataclass(eq=False)   # requests compare by identity: their point arrays do not compare
class Request:
    pts: np.ndarray
    want_residual: bool
    t_arrival: float = 0.0
    t_done: float = 0.0
    result: np.ndarray | None = None
    error: str | None = None
    rid: int = 0
    retries: int = 0
    cancelled: bool = False
    final: bool = False             # its outcome is being delivered: too late to cancel
    out: np.ndarray | None = None   # caller-owned result rows, filled in place
    done: threading.Event = field(default_factory=threading.Event)
    parent: "Request | None" = None  # a chunk of a request larger than a slot
    chunks: list = field(default_factory=list)
    remaining: int = 0

    @property
    def n(self) -> int:
        return int(self.pts.shape[0])

    @property
    def latency_ms(self) -> float:
        return 1e3 * (self.t_done - self.t_arrival)


def slot_bytes_per_point(d_in: int, w_val: int, w_res: int) -> int:
    """Device bytes per point of one slot's capacity: the points, the value
    and residual rows, and the routing scratch of the slot's two query
    contexts (net index and order: two ints per point each, plus at most one
    32-byte work item per 64 points each)."""
    return 4 * (d_in + w_val + w_res) + 2 * (8 + 1)


ALLOC_GRANULE = 2 << 20   # device allocations are counted rounded up to 2 MiB


def slot_fixed_bytes(n_nets: int) -> int:
    """Device bytes of one slot independent of its capacity: per-net counts,
    offsets and cursors and one work item per net in each query context, and
    the rounding of the slot's five device allocations (three buffers, one
    per query context) up to the allocation granule."""
    return 2 * (12 * n_nets + 32 * (n_nets + 1) + 8 * 256) + 5 * ALLOC_GRANULE


def request_bytes(n: int, d_in: int, width: int) -> int:
    """Device bytes a request holds while in flight: its points, its output
    rows and the routing scratch (net index and order, two ints per point)."""
    return n * 4 * (d_in + width + 2)


def plan_batch(pending, max_points: int, budget_left: int, d_in: int, width_of):
    """FIFO admission: the longest prefix of ``pending`` that fits both the
    slot's point capacity and the remaining memory budget.  Requests larger
    than a slot arrive here as slot-sized chunks (split at submission)."""
    take, pts, mem = [], 0, 0
    for r in pending:
        b = request_bytes(r.n, d_in, width_of(r))
        if pts + r.n > max_points or mem + b > budget_left:
            break
        take.append(r)
        pts += r.n
        mem += b
    return take, mem


class Server:
    """``mem_cap_bytes`` bounds all device memory the server allocates: the
    slots' capacity in points is the largest that fits ``slots`` slots under
    the cap (at most ``max_batch_points`` when given).  ``device_bytes`` is
    the resulting reservation."""

    def __init__(self, handle, slots: int = 4, mem_cap_bytes: int = 8 << 30, max_batch_points: int | None = 1 << 21):
        import torch
        from .binding import QueryContext
        self.torch = torch
        self.d = handle
        self.d_in, self.d_out, self.ds = handle.d_in, handle.d_out, handle.d_space
        self.w_val = self.d_out
        self.w_res = self.d_out + self.ds + 1
        self.mem_cap = int(mem_cap_bytes)
        per_pt = slot_bytes_per_point(self.d_in, self.w_val, self.w_res)
        fixed = slot_fixed_bytes(handle.n_nets)
        fit = (self.mem_cap // max(1, slots) - fixed) // per_pt
        self.max_points = int(min(fit, max_batch_points) if max_batch_points else fit)
        if self.max_points < 1024:
            raise ValueError(f"a memory cap of {self.mem_cap} bytes leaves fewer than 1024 points per slot")
        self.device_bytes = slots * (self.max_points * per_pt + fixed)
        cfg = handle.cfg
        self.lo = np.array([np.float32(cfg["lo"][a]) for a in range(self.d_in)], np.float32)
        self.hi = np.array([np.float32(cfg["hi"][a]) for a in range(self.d_in)], np.float32)
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                # lower numbers are higher priorities; out-of-range values map
                # to the nearest valid one (the highest for the value stream)
                "stream": torch.cuda.Stream(priority=-8),   # values
                "stream_r": torch.cuda.Stream(priority=0),  # residuals (the lowest)
                "qctx": QueryContext(handle, self.max_points),
                "qctx_r": QueryContext(handle, self.max_points),
                "pts_h": torch.empty((self.max_points, self.d_in), dtype=torch.float32).pin_memory(),
                "pts_d": torch.empty((self.max_points, self.d_in), dtype=torch.float32, device="cuda"),
                "val_d": torch.empty((self.max_points, self.w_val), dtype=torch.float32, device="cuda"),
                "res_d": torch.empty((self.max_points, self.w_res), dtype=torch.float32, device="cuda"),
                "val_h": torch.empty((self.max_points, self.w_val), dtype=torch.float32).pin_memory(),
                "res_h": torch.empty((self.max_points, self.w_res), dtype=torch.float32).pin_memory(),
                "busy": None,
            })
        self.pending = deque()
        self.lock = threading.Condition()
        self.in_flight_bytes = 0
        self.max_in_flight_bytes = 0
        self.max_concurrent = 0
        self.completed = []
        self._next_id = 0
        self._stop = False
        self._thread = None

    # -- client side ------------------------------------------------------
    def submit(self, pts: np.ndarray, want_residual: bool = False, out: np.ndarray | None = None) -> Request:
        """Queue a query of ``pts`` ([n][d_in]).  ``out``, if given, is a
        caller-owned float32 array [n][width] (width 4 or 8 as for the result)
        that receives the result in place (and becomes ``result``), so that a
        client can reuse its buffers instead of receiving a new array."""
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, self.d_in)
        r = Request(pts=pts, want_residual=bool(want_residual), t_arrival=time.perf_counter())
        if out is not None:
            if (not isinstance(out, np.ndarray) or out.dtype != np.float32 or
                    out.shape != (r.n, self._width(r))):
                raise ValueError(f"out must be a float32 array of shape ({r.n}, {self._width(r)})")
            r.out = out
        with self.lock:
            r.rid = self._next_id
            self._next_id += 1
        # The domain is checked on the device while routing; only a batch that
        # reports an outside point is checked request by request on the host
        # (see _complete), which keeps the check off the common path.
        if r.n == 0:
            r.result = np.zeros((0, self._width(r)), np.float32)
            r.t_done = time.perf_counter()
            r.done.set()
            return r
        if r.n > self.max_points:
            # larger than a slot: slot-sized chunks writing into rows of one
            # result, queued together; the request completes with its last chunk
            if r.out is None:
                r.out = np.empty((r.n, self._width(r)), np.float32)
            for a in range(0, r.n, self.max_points):
                b = min(r.n, a + self.max_points)
                r.chunks.append(Request(pts=r.pts[a:b], want_residual=r.want_residual, t_arrival=r.t_arrival,
                                        rid=r.rid, out=r.out[a:b], parent=r))
            r.remaining = len(r.chunks)
            with self.lock:
                self.pending.extend(r.chunks)
                self.lock.notify()
            return r
        with self.lock:
            self.pending.append(r)
            self.lock.notify()
        return r

    def _deliver(self, r: Request):
        """Completion of a request or chunk (outcome already set; the lock is
        held): a chunk completes its parent with the last of its chunks."""
        p = r.parent
        if p is None:
            r.done.set()
            self.completed.append(r)
            return
        if r.error and not p.error:
            p.error = r.error
        p.remaining -= 1
        if p.remaining == 0:
            p.t_done = max(c.t_done for c in p.chunks)
            p.final = True
            if not p.error:
                p.result = p.out
            p.done.set()
            self.completed.append(p)

    def cancel(self, r: Request) -> bool:
        """Withdraw a request: a waiting one leaves the queue at once; one
        already on the GPU finishes there but its result is dropped.  Both end
        with error "cancelled" (True); a finished request is left as it is
        (False)."""
        with self.lock:
            if r.done.is_set() or r.final:
                return False
            r.cancelled = True
            if r.chunks:   # every chunk: waiting ones leave the queue, running ones are dropped
                if all(c.final for c in r.chunks):
                    r.cancelled = False
                    return False
                r.error = "cancelled"
                for c in r.chunks:
                    if c.final or c.done.is_set():
                        continue
                    c.cancelled = True
                    if c in self.pending:
                        self.pending.remove(c)
                        c.error = "cancelled"
                        c.t_done = time.perf_counter()
                        self._deliver(c)
                return True
            if r in self.pending:
                self.pending.remove(r)
                r.error = "cancelled"
                r.t_done = time.perf_counter()
                r.done.set()
        return True

    def _width(self, r):
        return self.w_res if r.want_residual else self.w_val

    # -- dispatcher ----------------------------------------------------------
    def start(self):
        self._stop = False
        self._thread = threading.Thread(target=self._run, daemon=True)
        self._thread.start()
        return self

    def stop(self, drain: bool = True):
        if drain:
            while True:
                with self.lock:
                    if not self.pending and all(s["busy"] is None for s in self.slots):
                        break
                time.sleep(0.001)
        self._stop = True
        with self.lock:
            self.lock.notify()
        if self._thread:
            self._thread.join()
        for s in self.slots:
            s["qctx"].close()
            s["qctx_r"].close()

    def _run(self):
        torch = self.torch
        torch.cuda.set_device(self.d.cfg.get("device", 0))
        while not self._stop:
            progressed = self._complete()
            with self.lock:
                free = [s for s in self.slots if s["busy"] is None]
                batches = []
                for s in free:
                    take, mem = plan_batch(self.pending, self.max_points, self.mem_cap - self.in_flight_bytes,
                                           self.d_in, self._width)
                    if not take:
                        break
                    for _ in take:
                        self.pending.popleft()
                    self.in_flight_bytes += mem
                    self.max_in_flight_bytes = max(self.max_in_flight_bytes, self.in_flight_bytes)
                    batches.append((s, take, mem))
                if not batches and not progressed and all(s["busy"] is None for s in self.slots):
                    self.lock.wait(timeout=0.002)
            for s, take, mem in batches:
                self._launch(s, take, mem)
            busy = sum(1 for s in self.slots if s["busy"] is not None)
            self.max_concurrent = max(self.max_concurrent, busy)
            if not batches and not progressed:
                time.sleep(0.0002)

    def _launch(self, s, take, mem):
        torch = self.torch
        vals = [r for r in take if not r.want_residual]
        ress = [r for r in take if r.want_residual]
        order = vals + ress
        nv = sum(r.n for r in vals)
        nr = sum(r.n for r in ress)
        ph = s["pts_h"].numpy()
        off = 0
        for r in order:
            ph[off:off + r.n] = r.pts
            off += r.n
        stream, stream_r = s["stream"], s["stream_r"]
        ev_v = ev_r = None
        with torch.cuda.stream(stream):
            s["pts_d"][:off].copy_(s["pts_h"][:off], non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(stream)
            if nv:
                s["qctx"].query_into(s["pts_d"][:nv], s["val_d"][:nv], False, stream)
                s["val_h"][:nv].copy_(s["val_d"][:nv], non_blocking=True)
                ev_v = torch.cuda.Event()
                ev_v.record(stream)
        if nr:
            with torch.cuda.stream(stream_r):
                stream_r.wait_event(ev_in)
                s["qctx_r"].query_into(s["pts_d"][nv:off], s["res_d"][:nr], True, stream_r)
                s["res_h"][:nr].copy_(s["res_d"][:nr], non_blocking=True)
                ev_r = torch.cuda.Event()
                ev_r.record(stream_r)
        s["busy"] = {"ev_v": ev_v, "ev_r": ev_r, "vals": vals, "ress": ress, "mem": mem}

    def _complete(self):
        done_any = False
        for s in self.slots:
            b = s["busy"]
            if b is None:
                continue
            t = None
            # values and residuals of a batch complete on their own events
            for key_ev, key_reqs, qctx, stream, buf, w in (("ev_v", "vals", s["qctx"], s["stream"], "val_h", self.w_val),
                                                           ("ev_r", "ress", s["qctx_r"], s["stream_r"], "res_h",
                                                            self.w_res)):
                ev = b[key_ev]
                if ev is None or not ev.query():
                    continue
                st = qctx.status(stream)
                t = time.perf_counter()
                h = s[buf].numpy()
                finished, retry = [], []
                off = 0
                for r in b[key_reqs]:
                    with self.lock:   # decided once: a later cancel() returns False
                        cancelled = r.cancelled or (r.parent is not None and r.parent.cancelled)
                        r.final = True
                    if cancelled:
                        r.error = "cancelled"
                    elif st == 0:
                        if r.out is not None:
                            np.copyto(r.out, h[off:off + r.n])
                            r.result = r.out
                        else:
                            r.result = h[off:off + r.n].copy()
                    elif (st == ERR_INVALID_ARG and r.retries == 0 and
                          np.all((r.pts >= self.lo) & (r.pts <= self.hi))):
                        r.retries += 1       # an innocent neighbour of an outside point: run it again
                        with self.lock:
                            r.final = False
                        retry.append(r)
                        off += r.n
                        continue
                    else:
                        r.error = ("query point outside the domain" if st == ERR_INVALID_ARG
                                   else f"query failed with status {st}")
                    off += r.n
                    r.t_done = t
                    finished.append(r)
                with self.lock:
                    for r in finished:
                        self._deliver(r)
                    for r in reversed(retry):
                        self.pending.appendleft(r)
                b[key_ev] = None
                done_any = True
            if b["ev_v"] is None and b["ev_r"] is None:
                with self.lock:
                    self.in_flight_bytes -= b["mem"]
                    s["busy"] = None
        return done_any


def poisson_load(server: Server, cfg: dict, rate_hz: float, duration_s: float, seed: int = 0,
                 n_min: int = 1000, n_max: int = 1_000_000, residual_fraction: float = 0.1, pool=None,
                 client_buffers: bool = False):
    """Open-loop Poisson arrivals; each request a uniform space-time point cloud
    of log-uniform size (a slice of a pre-generated uniform pool, so that
    producing a request costs nothing), a fraction asking for residuals.
    With ``client_buffers`` every request gets its own rows of two result
    arrays allocated and touched before the first arrival (a client with its
    own output memory), so that results are written in place.
    Returns the requests once all are done."""
    from . import synth
    rng = np.random.default_rng(seed)
    if pool is None:
        pool = synth.query_points(cfg, 2 * n_max, seed=seed + 7)
    sched = []
    t = 0.0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        n = int(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        off = int(rng.integers(0, len(pool) - n + 1))
        sched.append((t, off, n, bool(rng.random() < residual_fraction)))
    outs = [None] * len(sched)
    if client_buffers:
        rows = {w: sum(n for (_, _, n, want) in sched if want == w) for w in (False, True)}
        ring = {w: np.empty((max(rows[w], 1), server.w_res if w else server.w_val), np.float32) for w in rows}
        pos = {False: 0, True: 0}
        for w in ring:
            ring[w].fill(0.0)   # touch every page now, not while serving
        for i, (_, _, n, want) in enumerate(sched):
            outs[i] = ring[want][pos[want]:pos[want] + n]
            pos[want] += n
    t0 = time.perf_counter()
    reqs = []
    for i, (ta, off, n, want) in enumerate(sched):
        while time.perf_counter() - t0 < ta:
            time.sleep(max(0.0, min(0.0005, ta - (time.perf_counter() - t0))))
        reqs.append(server.submit(pool[off:off + n], want, out=outs[i]))
    for r in reqs:
        r.done.wait()
    return reqs


def latency_summary(reqs):
    ok = [r for r in reqs if r.error is None]
    lat = np.array([r.latency_ms for r in ok]) if ok else np.zeros(1)
    pts = sum(r.n for r in ok)
    span = (max(r.t_done for r in ok) - min(r.t_arrival for r in ok)) if ok else 1.0
    return {"requests": len(reqs), "errors": len(reqs) - len(ok), "points": pts,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "points_per_s": pts / span if span > 0 else 0.0}
