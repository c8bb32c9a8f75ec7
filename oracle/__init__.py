"""ctypes binding of the FP64 CPU oracle (``oracle/oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check
and by the benchmark's CPU-baseline leg.  The product path never imports it.
All arrays cross the boundary as float64 (parameters, results) or as the very
float32 point arrays the CUDA path receives.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.cpp")


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, C++17, -O2)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               "-pthread", "-o", _SO, _SRC]
        subprocess.check_call(cmd)
    return _SO


class Config(C.Structure):
    _fields_ = [
        ("d_space", C.c_int), ("unsteady", C.c_int), ("depth", C.c_int), ("width", C.c_int),
        ("splits", C.c_int * 4), ("lo", C.c_double * 4), ("hi", C.c_double * 4),
        ("nu", C.c_double), ("anchor", C.c_double * 3), ("p_ref", C.c_double),
        ("lam_obs", C.c_double), ("lam_pde", C.c_double), ("lam_gh_u", C.c_double),
        ("lam_gh_p_space", C.c_double), ("lam_gh_p_time", C.c_double),
        ("comp_w", C.c_double * 3),
        ("lr", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps", C.c_double),
        ("clip", C.c_double),
        ("lr_decay_factor", C.c_double), ("lr_decay_interval", C.c_int), ("comm_interval", C.c_int),
        ("activation", C.c_int),
        ("lam_gh_r", C.c_double), ("lam_gh_c1", C.c_double),
    ]


NLOSS = 8   # obs, PDE, gh_u, gh_p space, gh_p time, total, gh_r (residual matching), gh_c1


class ProblemC(C.Structure):
    _fields_ = [
        ("res_pts", C.c_void_p), ("res_counts", C.c_void_p),
        ("obs_pts", C.c_void_p), ("obs_vals", C.c_void_p), ("obs_counts", C.c_void_p),
        ("face_pts", C.c_void_p), ("face_counts", C.c_void_p),
        ("ghost_pts", C.c_void_p), ("ghost_counts", C.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        sig = {
            "ora_set_threads": [i32],
            "ora_layout": [vp] * 8,
            "ora_forward": [vp, i32, vp, vp, i64, i32, vp],
            "ora_forward_complex": [vp, i32, vp, vp, vp, vp, i64, i32, vp, vp],
            "ora_residual": [vp, vp, i64, vp],
            "ora_forward_vjp": [vp, i32, vp, vp, i32, vp, vp],
            "ora_residual_vjp": [vp] * 4,
            "ora_exchange": [vp] * 5,
            "ora_losses": [vp] * 4,
            "ora_net_loss_complex": [vp, vp, vp, i32, vp, vp, vp, vp],
            "ora_grad_nets": [vp, vp, vp, vp, i32, vp, vp],
            "ora_grad": [vp] * 5,
            "ora_adam": [vp] * 6,
            "ora_step": [vp] * 7,
            "ora_query": [vp, vp, vp, i64, i32, vp, vp],
            "ora_step_cached": [vp] * 9,
            "ora_sample": [vp, C.c_uint64, i64, vp, vp],
            "ora_splitmix64_nth": [C.c_uint64, C.c_uint64],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = C.c_int if name != "ora_set_threads" else None
        _lib.ora_splitmix64_nth.restype = C.c_uint64
    return _lib


def splitmix64_nth(seed: int, n: int) -> int:
    """n-th output (n >= 1) of SplitMix64 seeded with ``seed``."""
    return int(lib().ora_splitmix64_nth(int(seed) & (2**64 - 1), int(n) & (2**64 - 1)))


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def _p(a):
    return a.ctypes.data if a is not None else None


def make_config(cfg: dict) -> Config:
    c = Config()
    c.d_space, c.unsteady = cfg["d_space"], cfg["unsteady"]
    c.depth, c.width = cfg["depth"], cfg["width"]
    for a in range(4):
        c.splits[a] = int(cfg["splits"][a])
        c.lo[a] = float(cfg["lo"][a])
        c.hi[a] = float(cfg["hi"][a])
    c.nu = cfg["nu"]
    for a in range(3):
        c.anchor[a] = float(cfg["anchor"][a])
        c.comp_w[a] = float(cfg["comp_w"][a])
    c.p_ref = cfg["p_ref"]
    c.lam_obs, c.lam_pde, c.lam_gh_u = cfg["lambda_obs"], cfg["lambda_pde"], cfg["lambda_gh_u"]
    c.lam_gh_p_space, c.lam_gh_p_time = cfg["lambda_gh_p_space"], cfg["lambda_gh_p_time"]
    c.lr, c.beta1, c.beta2, c.eps, c.clip = cfg["lr"], cfg["beta1"], cfg["beta2"], cfg["eps"], cfg["clip_norm"]
    c.lam_gh_r = float(cfg.get("lambda_gh_r", 0.0))
    c.lam_gh_c1 = float(cfg.get("lambda_gh_c1", 0.0))
    c.lr_decay_factor = float(cfg.get("lr_decay_factor", 1.0))
    c.lr_decay_interval = int(cfg.get("lr_decay_interval", 0))
    c.comm_interval = int(cfg.get("comm_interval", 1))
    c.activation = int(cfg.get("activation", 0))
    return c


class Oracle:
    """FP64 oracle bound to one configuration and (optionally) one problem."""

    def __init__(self, cfg: dict, problem=None):
        self.cfg = cfg
        self.c = make_config(cfg)
        L = lib()
        nn, nf, npar = C.c_int(), C.c_int(), C.c_int()
        L.ora_layout(C.addressof(self.c), C.addressof(nn), C.addressof(nf), C.addressof(npar), None, None, None, None)
        self.n_nets, self.n_faces, self.n_params = nn.value, nf.value, npar.value
        self.master = np.zeros(self.n_nets, np.int32)
        self.box_lo = np.zeros((self.n_nets, 4))
        self.box_hi = np.zeros((self.n_nets, 4))
        self.faces = np.zeros((max(self.n_faces, 1), 4), np.int32)
        L.ora_layout(C.addressof(self.c), None, None, None, _p(self.master), _p(self.box_lo),
                     _p(self.box_hi), _p(self.faces))
        self.faces = self.faces[: self.n_faces]
        self.d_space = cfg["d_space"]
        self.d_in = cfg["d_space"] + cfg["unsteady"]
        self.d_out = cfg["d_space"] + 1
        self.C = self.d_in + 2
        self._keep = []
        self.pc = None
        if problem is not None:
            self.set_problem(problem)

    # -- problem -----------------------------------------------------------
    def set_problem(self, pb):
        arrs = [np.ascontiguousarray(pb.res_pts, np.float32), np.ascontiguousarray(pb.res_counts, np.int64),
                np.ascontiguousarray(pb.obs_pts, np.float32), np.ascontiguousarray(pb.obs_vals, np.float32),
                np.ascontiguousarray(pb.obs_counts, np.int64), np.ascontiguousarray(pb.face_pts, np.float32),
                np.ascontiguousarray(pb.face_counts, np.int64)]
        gc = getattr(pb, "ghost_counts", None)
        if gc is not None:
            arrs += [np.ascontiguousarray(pb.ghost_pts, np.float32), np.ascontiguousarray(gc, np.int64)]
        self._keep = arrs
        ptrs = [a.ctypes.data for a in arrs] + ([None, None] if gc is None else [])
        self.pc = ProblemC(*ptrs)

    # -- pieces ------------------------------------------------------------
    def forward(self, net, th_net, x, jets=True):
        x = np.ascontiguousarray(x, np.float64).reshape(-1, self.d_in)
        th = np.ascontiguousarray(th_net, np.float64)
        nc = self.C if jets else 1
        out = np.zeros((len(x), self.d_out, nc))
        lib().ora_forward(C.addressof(self.c), net, _p(th), _p(x), len(x), int(jets), _p(out))
        return out

    def forward_complex(self, net, th_re, th_im, x_re, x_im, jets=True):
        x_re = np.ascontiguousarray(x_re, np.float64).reshape(-1, self.d_in)
        x_im = None if x_im is None else np.ascontiguousarray(x_im, np.float64).reshape(-1, self.d_in)
        th_re = np.ascontiguousarray(th_re, np.float64)
        th_im = None if th_im is None else np.ascontiguousarray(th_im, np.float64)
        nc = self.C if jets else 1
        o_re = np.zeros((len(x_re), self.d_out, nc))
        o_im = np.zeros_like(o_re)
        lib().ora_forward_complex(C.addressof(self.c), net, _p(th_re), _p(th_im), _p(x_re), _p(x_im),
                                  len(x_re), int(jets), _p(o_re), _p(o_im))
        return o_re + 1j * o_im

    def forward_vjp(self, net, th_net, x, Yb, jets=True):
        x = np.ascontiguousarray(x, np.float64).reshape(self.d_in)
        th = np.ascontiguousarray(th_net, np.float64)
        Yb = np.ascontiguousarray(Yb, np.float64)
        g = np.zeros(self.n_params)
        lib().ora_forward_vjp(C.addressof(self.c), net, _p(th), _p(x), int(jets), _p(Yb), _p(g))
        return g

    def residual(self, Y):
        Y = np.ascontiguousarray(Y, np.float64).reshape(-1, self.d_out, self.C)
        r = np.zeros((len(Y), self.d_space + 1))
        lib().ora_residual(C.addressof(self.c), _p(Y), len(Y), _p(r))
        return r

    def residual_vjp(self, Y, rb):
        Y = np.ascontiguousarray(Y, np.float64).reshape(self.d_out, self.C)
        rb = np.ascontiguousarray(rb, np.float64)
        Yb = np.zeros((self.d_out, self.C))
        lib().ora_residual_vjp(C.addressof(self.c), _p(Y), _p(rb), _p(Yb))
        return Yb

    # -- whole problem ----------------------------------------------------
    def exchange(self, th):
        th = np.ascontiguousarray(th, np.float64)
        n = int(np.sum(self._keep[6]))
        val = np.zeros((n, 2, self.d_out))
        anc = np.zeros((n, 2))
        lib().ora_exchange(C.addressof(self.c), C.addressof(self.pc), _p(th), _p(val), _p(anc))
        return val, anc

    def losses(self, th):
        th = np.ascontiguousarray(th, np.float64)
        out = np.zeros((self.n_nets, NLOSS))
        lib().ora_losses(C.addressof(self.c), C.addressof(self.pc), _p(th), _p(out))
        return out

    def net_loss_complex(self, th, net, th_im=None, thA=None):
        """Loss record of ``net`` with own parameters ``thA + i th_im``
        (``thA`` defaults to the net's block of ``th``); messages from ``th``."""
        th = np.ascontiguousarray(th, np.float64)
        th_im = None if th_im is None else np.ascontiguousarray(th_im, np.float64)
        thA = None if thA is None else np.ascontiguousarray(thA, np.float64)
        o_re, o_im = np.zeros(NLOSS), np.zeros(NLOSS)
        lib().ora_net_loss_complex(C.addressof(self.c), C.addressof(self.pc), _p(th), net, _p(thA), _p(th_im),
                                   _p(o_re), _p(o_im))
        return o_re + 1j * o_im

    def grad(self, th, nets=None):
        th = np.ascontiguousarray(th, np.float64)
        nets = np.arange(self.n_nets, dtype=np.int32) if nets is None else np.ascontiguousarray(nets, np.int32)
        g = np.zeros((len(nets), self.n_params))
        loss = np.zeros((len(nets), NLOSS))
        lib().ora_grad_nets(C.addressof(self.c), C.addressof(self.pc), _p(th), _p(nets), len(nets), _p(g), _p(loss))
        return g, loss

    def adam(self, th, m, v, t, grad):
        th, m, v = (np.array(a, np.float64) for a in (th, m, v))
        grad = np.ascontiguousarray(grad, np.float64)
        tt = C.c_int64(int(t))
        lib().ora_adam(C.addressof(self.c), _p(th), _p(m), _p(v), C.addressof(tt), _p(grad))
        return th, m, v, tt.value

    def step(self, th, m, v, t):
        th, m, v = (np.array(a, np.float64) for a in (th, m, v))
        tt = C.c_int64(int(t))
        loss = np.zeros((self.n_nets, NLOSS))
        lib().ora_step(C.addressof(self.c), C.addressof(self.pc), _p(th), _p(m), _p(v), C.addressof(tt), _p(loss))
        return th, m, v, tt.value, loss

    def step_cached(self, th, m, v, t, cache):
        """One iteration with the communication interval; ``cache`` is a dict
        holding the messages between calls (created on first use)."""
        th, m, v = (np.array(a, np.float64) for a in (th, m, v))
        n = int(np.sum(self._keep[6]))
        if "val" not in cache:
            cache["val"] = np.zeros((max(n, 1), 2, self.d_out))
            cache["anc"] = np.zeros((max(n, 1), 2))
        tt = C.c_int64(int(t))
        loss = np.zeros((self.n_nets, NLOSS))
        rc = lib().ora_step_cached(C.addressof(self.c), C.addressof(self.pc), _p(th), _p(m), _p(v), C.addressof(tt),
                              _p(loss), _p(cache["val"]), _p(cache["anc"]))
        if rc:
            raise ValueError("interface jet terms with a communication interval > 1 are not cached by the oracle")
        return th, m, v, tt.value, loss

    def sample(self, seed, t, counts):
        """Collocation points of step ``t`` (uniform per net cell, SplitMix64
        streams): float32 [sum counts][d_in], nets in order."""
        counts = np.ascontiguousarray(counts, np.int64)
        out = np.empty((int(counts.sum()), self.d_in), np.float32)
        lib().ora_sample(C.addressof(self.c), int(seed), int(t), counts.ctypes.data, out.ctypes.data)
        return out

    def query(self, th, pts, want_res=False):
        th = np.ascontiguousarray(th, np.float64)
        pts = np.ascontiguousarray(pts, np.float32).reshape(-1, self.d_in)
        w = self.d_out + (self.d_space + 1 if want_res else 0)
        out = np.zeros((len(pts), w))
        nets = np.zeros(len(pts), np.int32)
        st = lib().ora_query(C.addressof(self.c), _p(th), _p(pts), len(pts), int(want_res), _p(out), _p(nets))
        return out, nets, st
