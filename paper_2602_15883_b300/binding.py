"""ctypes binding of libdpinn (C ABI in ``include/dpinn.h``).

Argument marshalling only: every step of the training step and of the query
path runs in the library's CUDA kernels.  There is no CPU fallback - if the
library is missing or cannot be loaded, constructing ``Dpinn`` raises.
Arrays may be NumPy arrays (host memory) or torch tensors (host or device);
torch is used only for device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DPINN_LIB", os.path.join(HERE, "libdpinn.so"))

POINTS_RESIDUAL, POINTS_OBS, POINTS_FACE, POINTS_GHOST = 0, 1, 2, 3

ERRORS = {
    -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT", -6: "BUSY", -7: "STATE",
}

EXPORTS = (
    "dpinn_config_default", "dpinn_create", "dpinn_destroy", "dpinn_last_error", "dpinn_get_layout",
    "dpinn_net_info", "dpinn_face_info", "dpinn_set_points", "dpinn_step", "dpinn_eval_grad", "dpinn_loss",
    "dpinn_get_grad", "dpinn_query", "dpinn_query_status", "dpinn_get_state", "dpinn_set_state",
    "dpinn_apply_grad", "dpinn_launches_per_step", "dpinn_step_timed", "dpinn_query_static",
    "dpinn_eval_loss", "dpinn_set_params", "dpinn_set_schedule", "dpinn_get_schedule",
    "dpinn_qctx_create", "dpinn_qctx_destroy", "dpinn_qctx_query", "dpinn_qctx_status",
    "dpinn_set_resampling", "dpinn_get_points", "dpinn_set_partial_budget", "dpinn_loss_ext",
    "dpinn_set_points_async", "dpinn_selftest_wait", "dpinn_loss_async", "dpinn_probe_fp32",
    "dpinn_query_jets", "dpinn_set_precision", "dpinn_get_precision", "dpinn_tile_options", "dpinn_set_tiles",
    "dpinn_get_tiles", "dpinn_selftest_sincos",
)


class DpinnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dpinn error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Config(C.Structure):
    _fields_ = [
        ("d_space", C.c_int), ("unsteady", C.c_int),
        ("lo", C.c_double * 4), ("hi", C.c_double * 4), ("splits", C.c_int * 4),
        ("depth", C.c_int), ("width", C.c_int), ("activation", C.c_int),
        ("nu", C.c_double), ("anchor_x", C.c_double * 3), ("p_ref", C.c_double),
        ("lambda_obs", C.c_double), ("lambda_pde", C.c_double), ("lambda_gh_u", C.c_double),
        ("lambda_gh_p_space", C.c_double), ("lambda_gh_p_time", C.c_double),
        ("comp_w", C.c_double * 3),
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("clip_norm", C.c_double),
        ("seed", C.c_uint64), ("precision", C.c_int), ("device", C.c_int),
        ("lr_decay_factor", C.c_double), ("lr_decay_interval", C.c_int), ("comm_interval", C.c_int),
        ("lambda_gh_r", C.c_double), ("lambda_gh_c1", C.c_double),
    ]


class Layout(C.Structure):
    _fields_ = [("n_nets", C.c_int), ("n_faces", C.c_int), ("d_in", C.c_int), ("d_out", C.c_int),
                ("n_params", C.c_int), ("n_masters", C.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdpinn.so (raises OSError when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libdpinn.so not built at {path}: run paper_2602_15883_b300/build.py")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
    sig = {
        "dpinn_config_default": ([vp], i32),
        "dpinn_create": ([vp, vp], i32),
        "dpinn_destroy": ([vp], None),
        "dpinn_last_error": ([vp], C.c_char_p),
        "dpinn_get_layout": ([vp, vp], i32),
        "dpinn_net_info": ([vp, i32, vp, vp, vp], i32),
        "dpinn_face_info": ([vp, i32, vp, vp, vp, vp], i32),
        "dpinn_set_points": ([vp, i32, vp, vp, vp, i32], i32),
        "dpinn_step": ([vp, vp, i32], i32),
        "dpinn_eval_grad": ([vp, vp], i32),
        "dpinn_loss": ([vp, vp], i32),
        "dpinn_get_grad": ([vp, vp], i32),
        "dpinn_query": ([vp, vp, i64, i32, vp, vp], i32),
        "dpinn_query_jets": ([vp, vp, i64, vp, vp], i32),
        "dpinn_set_precision": ([vp, i32], i32),
        "dpinn_get_precision": ([vp, vp], i32),
        "dpinn_tile_options": ([vp, vp, vp, vp, vp], i32),
        "dpinn_set_tiles": ([vp, i32, i32], i32),
        "dpinn_get_tiles": ([vp, vp, vp], i32),
        "dpinn_query_status": ([vp, vp], i32),
        "dpinn_get_state": ([vp, vp, vp, vp, vp], i32),
        "dpinn_set_state": ([vp, vp, vp, vp, i64], i32),
        "dpinn_apply_grad": ([vp, vp], i32),
        "dpinn_launches_per_step": ([vp], i32),
        "dpinn_step_timed": ([vp, vp, vp, i32, vp, vp], i32),
        "dpinn_query_static": ([vp, vp, i64, i32, vp, vp], i32),
        "dpinn_eval_loss": ([vp, vp], i32),
        "dpinn_set_params": ([vp, vp], i32),
        "dpinn_set_schedule": ([vp, i32, i32, i32], i32),
        "dpinn_get_schedule": ([vp, vp, vp, vp, vp], i32),
        "dpinn_qctx_create": ([vp, i64, vp], i32),
        "dpinn_qctx_destroy": ([vp], None),
        "dpinn_qctx_query": ([vp, vp, i64, i32, vp, vp], i32),
        "dpinn_qctx_status": ([vp, vp], i32),
        "dpinn_set_resampling": ([vp, vp, i32, C.c_uint64], i32),
        "dpinn_get_points": ([vp, i32, vp], i32),
        "dpinn_set_partial_budget": ([vp, i64], i32),
        "dpinn_loss_ext": ([vp, vp], i32),
        "dpinn_set_points_async": ([vp, i32, vp, vp, i32, vp], i32),
        "dpinn_selftest_wait": ([vp], i32),
        "dpinn_loss_async": ([vp, vp, vp], i32),
        "dpinn_probe_fp32": ([i32, i32, i64, vp, vp], i32),
        "dpinn_selftest_sincos": ([i32, vp, i64, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def make_config(cfg: dict) -> Config:
    c = Config()
    load_library().dpinn_config_default(C.addressof(c))
    c.d_space, c.unsteady = int(cfg["d_space"]), int(cfg["unsteady"])
    for a in range(4):
        c.lo[a] = float(cfg["lo"][a])
        c.hi[a] = float(cfg["hi"][a])
        c.splits[a] = int(cfg["splits"][a])
    c.depth, c.width = int(cfg["depth"]), int(cfg["width"])
    c.activation = int(cfg.get("activation", 0))
    c.nu = float(cfg["nu"])
    for a in range(3):
        c.anchor_x[a] = float(cfg["anchor"][a])
        c.comp_w[a] = float(cfg["comp_w"][a])
    c.p_ref = float(cfg["p_ref"])
    for k in ("lambda_obs", "lambda_pde", "lambda_gh_u", "lambda_gh_p_space", "lambda_gh_p_time",
              "lr", "beta1", "beta2", "eps", "clip_norm"):
        setattr(c, k, float(cfg[k]))
    c.seed = int(cfg.get("seed", 0))
    c.precision = int(cfg.get("precision", 0))
    c.device = int(cfg.get("device", 0))
    c.lr_decay_factor = float(cfg.get("lr_decay_factor", 1.0))
    c.lr_decay_interval = int(cfg.get("lr_decay_interval", 0))
    c.comm_interval = int(cfg.get("comm_interval", 1))
    c.lambda_gh_r = float(cfg.get("lambda_gh_r", 0.0))
    c.lambda_gh_c1 = float(cfg.get("lambda_gh_c1", 0.0))
    return c


def probe_fp32(iters, blocks_per_sm=4, device=0):
    """(milliseconds, FLOP) of one launch of the library's packed-FMA chain
    probe (dpinn_probe_fp32): the attainable FP32 FMA rate is FLOP / time."""
    lib = load_library()
    ms, flop = C.c_float(), C.c_double()
    rc = lib.dpinn_probe_fp32(int(device), int(blocks_per_sm), int(iters), C.byref(ms), C.byref(flop))
    if rc:
        raise DpinnError(rc, "dpinn_probe_fp32 failed")
    return ms.value, flop.value


def selftest_sincos(x):
    """(sin x, cos x) as the sin-activation kernels evaluate them
    (dpinn_selftest_sincos); x: a float32 CUDA tensor, returns an [n][2]
    float32 CUDA tensor on the same device."""
    import torch
    lib = load_library()
    x = x.contiguous()
    assert x.is_cuda and x.dtype == torch.float32
    out = torch.empty((x.numel(), 2), dtype=torch.float32, device=x.device)
    rc = lib.dpinn_selftest_sincos(int(x.device.index or 0), C.c_void_p(x.data_ptr()), int(x.numel()),
                                   C.c_void_p(out.data_ptr()))
    if rc:
        raise DpinnError(rc, "dpinn_selftest_sincos failed")
    return out


def _ptr(a):
    """(pointer, keep-alive) for a NumPy array or a torch tensor."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, a
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.contiguous()
            return a.data_ptr(), a
    except ImportError:
        pass
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Dpinn:
    """One resident ensemble of subdomain networks on one GPU."""

    def __init__(self, cfg: dict):
        self.lib = load_library()
        self.cfg = dict(cfg)
        self._c = make_config(cfg)
        h = C.c_void_p()
        rc = self.lib.dpinn_create(C.addressof(self._c), C.addressof(h))
        if rc != 0:
            raise DpinnError(rc, self.lib.dpinn_last_error(None).decode())
        self.h = h
        lay = Layout()
        self._check(self.lib.dpinn_get_layout(self.h, C.addressof(lay)))
        self.n_nets, self.n_faces = lay.n_nets, lay.n_faces
        self.d_in, self.d_out, self.n_params = lay.d_in, lay.d_out, lay.n_params
        self.n_masters = lay.n_masters
        self.d_space = self.d_out - 1

    def _check(self, rc):
        if rc != 0:
            raise DpinnError(rc, self.lib.dpinn_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.dpinn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout -------------------------------------------------------------
    def net_info(self, k):
        m = C.c_int()
        lo = (C.c_double * 4)()
        hi = (C.c_double * 4)()
        self._check(self.lib.dpinn_net_info(self.h, k, C.addressof(m), C.addressof(lo), C.addressof(hi)))
        return m.value, np.array(lo[:]), np.array(hi[:])

    def face_info(self, f):
        v = [C.c_int() for _ in range(4)]
        self._check(self.lib.dpinn_face_info(self.h, f, *[C.addressof(x) for x in v]))
        return tuple(x.value for x in v)

    # -- points ---------------------------------------------------------------
    def set_points(self, kind, pts, counts, vals=None):
        counts = np.ascontiguousarray(counts, np.int64)
        p, kp = _ptr(pts)
        q, kq = _ptr(vals)
        self._check(self.lib.dpinn_set_points(self.h, kind, p, q, counts.ctypes.data, len(counts)))

    def set_points_async(self, kind, pts, counts, stream=None):
        """Upload the next step's residual points asynchronously (``pts``
        pinned host memory kept unchanged until that step has completed)."""
        counts = np.ascontiguousarray(counts, np.int64)
        p, keep = _ptr(pts)
        if keep is not pts:   # a temporary copy would not outlive the copy in flight
            return self.set_points(kind, pts, counts)
        self._check(self.lib.dpinn_set_points_async(self.h, kind, p, counts.ctypes.data, len(counts),
                                                    _stream(stream)))

    def set_resampling(self, counts, seed=0):
        """Fresh uniform residual points in every net's cell before each step
        (``counts`` per net), or off with ``counts=None``."""
        if counts is None:
            self._check(self.lib.dpinn_set_resampling(self.h, None, 0, 0))
            return
        counts = np.ascontiguousarray(counts, np.int64)
        self._check(self.lib.dpinn_set_resampling(self.h, counts.ctypes.data, len(counts), int(seed)))
        self._res_counts = counts.copy()

    def get_points(self, kind, n):
        """The current points of a set as float32 [n][d_in] (n = sum of its counts)."""
        out = np.empty((int(n), self.d_in), np.float32)
        self._check(self.lib.dpinn_get_points(self.h, int(kind), out.ctypes.data))
        return out

    def set_partial_budget(self, nbytes):
        self._check(self.lib.dpinn_set_partial_budget(self.h, int(nbytes)))

    def set_problem(self, pb, set_params=True):
        self.set_points(POINTS_RESIDUAL, np.asarray(pb.res_pts, np.float32), pb.res_counts)
        self.set_points(POINTS_OBS, np.asarray(pb.obs_pts, np.float32), pb.obs_counts,
                        np.asarray(pb.obs_vals, np.float32))
        if getattr(pb, "ghost_counts", None) is not None:
            self.set_points(POINTS_GHOST, np.asarray(pb.ghost_pts, np.float32), pb.ghost_counts)
        else:
            self.set_points(POINTS_FACE, np.asarray(pb.face_pts, np.float32), pb.face_counts)
        if set_params:
            self.set_state(params=pb.theta0, step=0, zero_moments=True)

    # -- training -------------------------------------------------------------
    def step(self, n=1, stream=None):
        self._check(self.lib.dpinn_step(self.h, _stream(stream), int(n)))

    def eval_grad(self, stream=None):
        self._check(self.lib.dpinn_eval_grad(self.h, _stream(stream)))

    def eval_loss(self, stream=None):
        self._check(self.lib.dpinn_eval_loss(self.h, _stream(stream)))

    def set_params(self, params):
        """Replace the parameters (NumPy or torch, host or device) only."""
        p, keep = _ptr(params)
        self._check(self.lib.dpinn_set_params(self.h, p))

    def grad_into(self, out):
        """Copy the last gradient into a torch tensor / NumPy array (any device)."""
        p, keep = _ptr(out)
        self._check(self.lib.dpinn_get_grad(self.h, p))
        return out

    def loss(self, check=True):
        out = np.zeros((self.n_nets, 6), np.float32)
        rc = self.lib.dpinn_loss(self.h, out.ctypes.data)
        if check:
            self._check(rc)
        return out

    def loss_async(self, out, stream=None):
        """Queue a copy of the loss record [n_nets][6] into ``out`` (a pinned
        float32 host tensor or array owned by the caller) on ``stream`` and
        return at once; ``out`` is valid once the stream reaches this point."""
        p, keep = _ptr(out)
        if keep is not out or tuple(out.shape) != (self.n_nets, 6) or str(out.dtype) not in ("float32",
                                                                                               "torch.float32"):
            raise ValueError("loss_async needs a contiguous float32 [n_nets][6] host buffer")
        if getattr(out, "is_cuda", False):
            raise ValueError("loss_async writes host memory")
        self._check(self.lib.dpinn_loss_async(self.h, p, _stream(stream)))

    def loss_ext(self, check=True):
        """Loss record with the interface terms: [n_nets][8] (L_obs, L_PDE,
        L_gh_u, L_gh_p space, L_gh_p time, L_total, L_gh_r, L_gh_c1)."""
        out = np.zeros((self.n_nets, 8), np.float32)
        rc = self.lib.dpinn_loss_ext(self.h, out.ctypes.data)
        if check:
            self._check(rc)
        return out

    def grad(self):
        out = np.zeros((self.n_nets, self.n_params), np.float32)
        self._check(self.lib.dpinn_get_grad(self.h, out.ctypes.data))
        return out

    def get_state(self):
        n = self.n_nets * self.n_params
        th, m, v = (np.zeros(n, np.float32) for _ in range(3))
        st = C.c_int64()
        self._check(self.lib.dpinn_get_state(self.h, th.ctypes.data, m.ctypes.data, v.ctypes.data,
                                             C.addressof(st)))
        return th, m, v, st.value

    def set_state(self, params=None, m=None, v=None, step=0, zero_moments=False):
        n = self.n_nets * self.n_params
        if zero_moments:
            m = np.zeros(n, np.float32) if m is None else m
            v = np.zeros(n, np.float32) if v is None else v
        arrs = [None if a is None else np.ascontiguousarray(a, np.float32).reshape(-1) for a in (params, m, v)]
        for a in arrs:
            if a is not None and a.size != n:
                raise ValueError(f"state arrays need {n} floats, got {a.size}")
        ptrs = [None if a is None else a.ctypes.data for a in arrs]
        self._check(self.lib.dpinn_set_state(self.h, *ptrs, int(step)))

    def apply_grad(self, g):
        g = np.ascontiguousarray(g, np.float32).reshape(-1)
        self._check(self.lib.dpinn_apply_grad(self.h, g.ctypes.data))

    def step_timed(self, stream=None):
        """One step launched kernel by kernel with CUDA events between them:
        {kernel name: milliseconds}."""
        ms = (C.c_float * 8)()
        names = (C.c_char_p * 8)()
        n = C.c_int()
        self._check(self.lib.dpinn_step_timed(self.h, _stream(stream), C.addressof(ms), 8, C.addressof(n),
                                              C.addressof(names)))
        return {names[i].decode(): ms[i] for i in range(n.value)}

    def set_schedule(self, jet_tiles=0, val_tiles=0, order=0):
        self._check(self.lib.dpinn_set_schedule(self.h, int(jet_tiles), int(val_tiles), int(order)))

    def set_precision(self, precision):
        """Switch the contraction arithmetic (0 FP32, 1 TF32x3 at width 128)."""
        self._check(self.lib.dpinn_set_precision(self.h, int(precision)))
        self.cfg = dict(self.cfg, precision=int(precision))

    def tile_options(self):
        """(jet tile sizes, value tile sizes) in points, default first."""
        jo, vo = (C.c_int * 2)(), (C.c_int * 2)()
        nj, nv = C.c_int(), C.c_int()
        self._check(self.lib.dpinn_tile_options(self.h, jo, C.addressof(nj), vo, C.addressof(nv)))
        return list(jo[:nj.value]), list(vo[:nv.value])

    def set_tiles(self, jet_tile=0, val_tile=0):
        """Select the register tiles by index into tile_options() (0 = default)."""
        self._check(self.lib.dpinn_set_tiles(self.h, int(jet_tile), int(val_tile)))

    def get_tiles(self):
        j, v = C.c_int(), C.c_int()
        self._check(self.lib.dpinn_get_tiles(self.h, C.addressof(j), C.addressof(v)))
        return j.value, v.value

    def get_precision(self):
        p = C.c_int()
        self._check(self.lib.dpinn_get_precision(self.h, C.addressof(p)))
        return p.value

    def get_schedule(self):
        v = [C.c_int() for _ in range(3)]
        tp = (C.c_int * 2)()
        self._check(self.lib.dpinn_get_schedule(self.h, *[C.addressof(x) for x in v], C.addressof(tp)))
        return {"jet_tiles": v[0].value, "val_tiles": v[1].value, "order": v[2].value,
                "tile_points": (tp[0], tp[1])}

    @property
    def launches_per_step(self):
        return self.lib.dpinn_launches_per_step(self.h)

    # -- queries --------------------------------------------------------------
    def query(self, pts, want_residual=False, out=None, stream=None, check=True):
        """Evaluate the ensemble at device points (torch CUDA tensor [n][d_in])."""
        import torch
        n = pts.shape[0]
        w = self.d_out + (self.d_space + 1 if want_residual else 0)
        if out is None:
            out = torch.empty((n, w), dtype=torch.float32, device=pts.device)
        p, kp = _ptr(pts)
        o, ko = _ptr(out)
        s = _stream(stream)
        self._check(self.lib.dpinn_query(self.h, p, n, int(bool(want_residual)), o, s))
        if check:
            self._check(self.lib.dpinn_query_status(self.h, s))
        return out

    def query_jets(self, pts, out=None, stream=None, check=True):
        """Raw output jets of the routed nets at device points: [n][d_out][d_in + 2]
        (channels: value, d/dx_q for every input, spatial Laplacian)."""
        import torch
        n = pts.shape[0]
        C = self.d_in + 2
        if out is None:
            out = torch.empty((n, self.d_out, C), dtype=torch.float32, device=pts.device)
        p, kp = _ptr(pts)
        o, ko = _ptr(out)
        s = _stream(stream)
        self._check(self.lib.dpinn_query_jets(self.h, p, n, o, s))
        if check:
            self._check(self.lib.dpinn_query_status(self.h, s))
        return out

    def query_status(self, stream=None):
        return self.lib.dpinn_query_status(self.h, _stream(stream))


class QueryContext:
    """Routing scratch for up to ``max_points`` points per query, so that
    queries through different contexts can be in flight on different streams."""

    def __init__(self, d: Dpinn, max_points: int):
        self.d = d
        q = C.c_void_p()
        d._check(d.lib.dpinn_qctx_create(d.h, int(max_points), C.addressof(q)))
        self.q = q
        self.max_points = int(max_points)

    def query_into(self, pts, out, want_residual=False, stream=None):
        p, kp = _ptr(pts)
        o, ko = _ptr(out)
        self.d._check(self.d.lib.dpinn_qctx_query(self.q, p, int(pts.shape[0]), int(bool(want_residual)), o,
                                                  _stream(stream)))
        return out

    def status(self, stream=None):
        return self.d.lib.dpinn_qctx_status(self.q, _stream(stream))

    def close(self):
        if getattr(self, "q", None):
            self.d.lib.dpinn_qctx_destroy(self.q)
            self.q = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
