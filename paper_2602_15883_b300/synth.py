"""Seeded synthetic workloads for the domain-decomposed PINN training step.

This module only *generates inputs*: collocation points, sparse noisy velocity
observations, interface (face) points and initial weights.  It holds none of
the method's arithmetic (no network, no residual, no loss), so that the CUDA
path and the FP64 oracle can both consume the very same arrays without sharing
any code that computes a result.

The paper's CFD datasets (lid-driven cavity, 2D/3D cylinder wakes) are not
available, so analytic incompressible flows stand in for them:

* Kovasznay flow (steady 2D, Re = 40),
* the decaying Taylor-Green vortex (unsteady 2D),
* the Ethier-Steinman Beltrami flow (unsteady 3D, a = pi/4, d = pi/2, nu = 1).

Their closed forms only produce the observation values; the physics residual
never sees them.

Array formats (shared with ``include/dpinn.h``):

* input coordinates are ``float32 [n][d_in]`` with the spatial axes first and
  time last (``d_in = d_space + unsteady``);
* nets are numbered over the cell grid with axis 0 fastest;
* faces are enumerated axis by axis (ascending), and within an axis by the
  lower net's id (ascending); a face joins net ``k`` and ``k + stride[axis]``;
* the per-net parameter block is, for each affine map ``l = 0..L``, the weight
  ``[out][in]`` row-major followed by the bias ``[out]``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

# Loss weights follow the paper's Table B1 (Appendix B):
# (lambda_obs, lambda_PDE, lambda_gh_u, lambda_gh_p) = (10, 4, 1, 1) for the
# steady 2D case, (10, 5, 1, 1) for the unsteady 2D case and (10, 10, 1, 1)
# for the unsteady 3D case.  The pressure ghost weight is used for both the
# spatial (base) and the temporal interfaces.


def _base(**kw):
    cfg = dict(
        d_space=2, unsteady=0, lo=[0.0] * 4, hi=[1.0] * 4, splits=[1] * 4,
        depth=4, width=32, activation=0, nu=0.01, anchor=[0.0, 0.0, 0.0],
        p_ref=0.0, lambda_obs=10.0, lambda_pde=4.0, lambda_gh_u=1.0,
        lambda_gh_p_space=1.0, lambda_gh_p_time=1.0, comp_w=[1.0, 1.0, 1.0],
        lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, clip_norm=0.0, seed=0,
        precision=0, device=0, lr_decay_factor=1.0, lr_decay_interval=0, comm_interval=1,
        # workload (not part of the library config)
        flow="kovasznay", res_dist=("const", 1000), n_obs=200, noise=0.01,
        n_face=0,
    )
    cfg.update(kw)
    return cfg


CONFIGS = {
    # Kovasznay, Re = 40, one 4 x 32 tanh net, 1,000 residual points,
    # 200 noisy (1 %) velocity measurements, anchor p(0,0).
    "kovasznay": _base(
        d_space=2, unsteady=0, lo=[-0.5, -0.5, 0, 0], hi=[1.0, 1.5, 0, 0],
        splits=[1, 1, 1, 1], depth=4, width=32, nu=1.0 / 40.0,
        anchor=[0.0, 0.0, 0.0], lambda_obs=10.0, lambda_pde=4.0,
        flow="kovasznay", res_dist=("const", 1000), n_obs=200, noise=0.01,
        n_face=0),
    # Taylor-Green vortex, nu = 0.01, [0, 2pi]^2 x [0, 1], 4 x 4 x 2 nets of
    # 6 x 64, 8,192 residual + 1,024 obs (1 %) per net, 512 points per face.
    "tgv": _base(
        d_space=2, unsteady=1, lo=[0.0, 0.0, 0.0, 0], hi=[2 * math.pi, 2 * math.pi, 1.0, 0],
        splits=[4, 4, 2, 1], depth=6, width=64, nu=0.01,
        anchor=[math.pi / 4, math.pi / 4, 0.0], lambda_obs=10.0, lambda_pde=5.0,
        flow="tgv", res_dist=("const", 8192), n_obs=1024, noise=0.01,
        n_face=512),
    # Beltrami, [-1, 1]^3 x [0, 1], 2 x 2 x 2 x 4 nets of 8 x 128, residual
    # points per net log-uniform in [4096, 32768], 2,048 obs (2 %), 1,024
    # points per face.
    "beltrami32": _base(
        d_space=3, unsteady=1, lo=[-1.0, -1.0, -1.0, 0.0], hi=[1.0, 1.0, 1.0, 1.0],
        splits=[2, 2, 2, 4], depth=8, width=128, nu=1.0,
        anchor=[-0.5, -0.5, -0.5], lambda_obs=10.0, lambda_pde=10.0,
        flow="beltrami", res_dist=("loguniform", 4096, 32768), n_obs=2048,
        noise=0.02, n_face=1024),
    # Beltrami, 4 x 4 x 2 x 4 = 128 nets of 6 x 128, residual points per net
    # from a truncated power law p(n) ~ n^-1.2 on [2048, 65536].
    "beltrami128": _base(
        d_space=3, unsteady=1, lo=[-1.0, -1.0, -1.0, 0.0], hi=[1.0, 1.0, 1.0, 1.0],
        splits=[4, 4, 2, 4], depth=6, width=128, nu=1.0,
        anchor=[-0.75, -0.75, -0.5], lambda_obs=10.0, lambda_pde=10.0,
        flow="beltrami", res_dist=("powerlaw", 2048, 65536, 1.2), n_obs=2048,
        noise=0.02, n_face=1024),
    # The network shapes and point budgets of the paper's cylinder cases
    # (Sec. 5, Table B1) on analytic stand-in flows (the CFD data are not
    # available): 2-D, 6 x 150 sin, 5e5 residual and 1e4 observation points,
    # 1,000 points per interface, 4 x 2 (space x time) subdomains on the TGV
    # domain; 3-D, 8 x 200 sin, 6e5 residual and 1e5 observation points,
    # 5,000 points per interface, 2 x 2 x 1 x 2 subdomains on the Beltrami
    # domain.
    "cylinder2d": _base(
        d_space=2, unsteady=1, lo=[0.0, 0.0, 0.0, 0], hi=[2 * math.pi, 2 * math.pi, 1.0, 0],
        splits=[4, 1, 2, 1], depth=6, width=150, activation=1, nu=0.01,
        anchor=[math.pi / 4, math.pi / 4, 0.0], lambda_obs=10.0, lambda_pde=5.0,
        flow="tgv", res_dist=("const", 62500), n_obs=1250, noise=0.01,
        n_face=1000),
    "cylinder3d": _base(
        d_space=3, unsteady=1, lo=[-1.0, -1.0, -1.0, 0.0], hi=[1.0, 1.0, 1.0, 1.0],
        splits=[2, 2, 1, 2], depth=8, width=200, activation=1, nu=1.0,
        anchor=[-0.5, -0.5, -0.5], lambda_obs=10.0, lambda_pde=10.0,
        flow="beltrami", res_dist=("const", 75000), n_obs=12500, noise=0.02,
        n_face=5000),
}

LIB_KEYS = (
    "d_space", "unsteady", "lo", "hi", "splits", "depth", "width", "activation",
    "nu", "anchor", "p_ref", "lambda_obs", "lambda_pde", "lambda_gh_u",
    "lambda_gh_p_space", "lambda_gh_p_time", "comp_w", "lr", "beta1", "beta2",
    "eps", "clip_norm", "seed", "precision", "device", "lr_decay_factor", "lr_decay_interval",
    "comm_interval",
)


def config(name: str, **overrides) -> dict:
    """A copy of a named workload configuration with ``overrides`` applied."""
    cfg = {k: (list(v) if isinstance(v, list) else v) for k, v in CONFIGS[name].items()}
    cfg.update(overrides)
    return cfg


# --------------------------------------------------------------------------
# geometry of the decomposition (only what sampling needs)
# --------------------------------------------------------------------------

def d_in(cfg) -> int:
    return cfg["d_space"] + cfg["unsteady"]


def d_out(cfg) -> int:
    return cfg["d_space"] + 1


def n_nets(cfg) -> int:
    return int(np.prod(cfg["splits"][: d_in(cfg)]))


def strides(cfg):
    s, out = 1, []
    for a in range(d_in(cfg)):
        out.append(s)
        s *= cfg["splits"][a]
    return out


def cell_of_net(cfg, k):
    c = []
    for a in range(d_in(cfg)):
        c.append(k % cfg["splits"][a])
        k //= cfg["splits"][a]
    return c


def net_box(cfg, k):
    """Return (lo, hi) float64 arrays of net ``k``'s interior cell."""
    c = cell_of_net(cfg, k)
    lo, hi = [], []
    for a in range(d_in(cfg)):
        h = (cfg["hi"][a] - cfg["lo"][a]) / cfg["splits"][a]
        lo.append(cfg["lo"][a] + c[a] * h)
        hi.append(cfg["lo"][a] + (c[a] + 1) * h)
    return np.array(lo), np.array(hi)


def faces(cfg):
    """List of (net_lo, net_hi, axis) in the canonical face order."""
    out = []
    st = strides(cfg)
    for a in range(d_in(cfg)):
        for k in range(n_nets(cfg)):
            if cell_of_net(cfg, k)[a] < cfg["splits"][a] - 1:
                out.append((k, k + st[a], a))
    return out


def n_params_net(cfg) -> int:
    W, L, di, do = cfg["width"], cfg["depth"], d_in(cfg), d_out(cfg)
    return W * di + W + (L - 1) * (W * W + W) + do * W + do


def layer_shapes(cfg):
    W, L, di, do = cfg["width"], cfg["depth"], d_in(cfg), d_out(cfg)
    shapes = [(W, di)] + [(W, W)] * (L - 1) + [(do, W)]
    return shapes


# --------------------------------------------------------------------------
# analytic flows (observation values only)
# --------------------------------------------------------------------------

def kovasznay(x, y, Re=40.0):
    lam = Re / 2.0 - math.sqrt(Re * Re / 4.0 + 4.0 * math.pi ** 2)
    e = np.exp(lam * x)
    u = 1.0 - e * np.cos(2 * math.pi * y)
    v = lam / (2 * math.pi) * e * np.sin(2 * math.pi * y)
    p = 0.5 * (1.0 - np.exp(2 * lam * x))
    return np.stack([u, v, p], -1)


def taylor_green(x, y, t, nu=0.01):
    f = np.exp(-2 * nu * t)
    u = np.cos(x) * np.sin(y) * f
    v = -np.sin(x) * np.cos(y) * f
    p = -0.25 * (np.cos(2 * x) + np.cos(2 * y)) * f * f
    return np.stack([u, v, p], -1)


def beltrami(x, y, z, t, a=math.pi / 4, d=math.pi / 2, nu=1.0):
    F = np.exp(-nu * d * d * t)
    u = -a * (np.exp(a * x) * np.sin(a * y + d * z) + np.exp(a * z) * np.cos(a * x + d * y)) * F
    v = -a * (np.exp(a * y) * np.sin(a * z + d * x) + np.exp(a * x) * np.cos(a * y + d * z)) * F
    w = -a * (np.exp(a * z) * np.sin(a * x + d * y) + np.exp(a * y) * np.cos(a * z + d * x)) * F
    p = -0.5 * a * a * F * F * (
        np.exp(2 * a * x) + np.exp(2 * a * y) + np.exp(2 * a * z)
        + 2 * np.sin(a * x + d * y) * np.cos(a * z + d * x) * np.exp(a * (y + z))
        + 2 * np.sin(a * y + d * z) * np.cos(a * x + d * y) * np.exp(a * (z + x))
        + 2 * np.sin(a * z + d * x) * np.cos(a * y + d * z) * np.exp(a * (x + y)))
    return np.stack([u, v, w, p], -1)


def flow_values(cfg, pts):
    """Analytic (u, v, [w], p) at float64 points ``[n][d_in]``."""
    pts = np.asarray(pts, np.float64)
    t = pts[:, cfg["d_space"]] if cfg["unsteady"] else np.zeros(len(pts))
    if cfg["flow"] == "kovasznay":
        return kovasznay(pts[:, 0], pts[:, 1], Re=1.0 / cfg["nu"])
    if cfg["flow"] == "tgv":
        return taylor_green(pts[:, 0], pts[:, 1], t, nu=cfg["nu"])
    if cfg["flow"] == "beltrami":
        return beltrami(pts[:, 0], pts[:, 1], pts[:, 2], t, nu=cfg["nu"])
    raise ValueError(cfg["flow"])


# --------------------------------------------------------------------------
# sampling
# --------------------------------------------------------------------------

def _rng(seed, *stream):
    return np.random.default_rng(np.random.SeedSequence([int(seed), *[int(s) for s in stream]]))


def residual_counts(cfg, seed=0):
    """Per-net collocation counts drawn from the configuration's distribution."""
    dist = cfg["res_dist"]
    n = n_nets(cfg)
    if dist[0] == "const":
        return np.full(n, int(dist[1]), np.int64)
    g = _rng(seed, 1)
    if dist[0] == "loguniform":
        lo, hi = math.log(dist[1]), math.log(dist[2])
        return np.rint(np.exp(g.uniform(lo, hi, n))).astype(np.int64)
    if dist[0] == "powerlaw":
        # truncated continuous power law p(n) ~ n^-s on [a, b], inverse CDF
        a, b, s = float(dist[1]), float(dist[2]), float(dist[3])
        u = g.uniform(0.0, 1.0, n)
        e = 1.0 - s
        vals = (a ** e + u * (b ** e - a ** e)) ** (1.0 / e)
        return np.rint(vals).astype(np.int64)
    if dist[0] == "list":
        return np.asarray(dist[1], np.int64)
    raise ValueError(dist)


def _uniform_in_box(g, lo, hi, n):
    return lo[None, :] + (hi - lo)[None, :] * g.uniform(0.0, 1.0, (n, lo.size))


def init_params(cfg, seed=0, bias_std=0.0):
    """Xavier-normal weights (std = sqrt(2/(fan_in+fan_out))), biases N(0, bias_std)."""
    out = []
    for k in range(n_nets(cfg)):
        g = _rng(seed, 5, k)
        for (fo, fi) in layer_shapes(cfg):
            std = math.sqrt(2.0 / (fi + fo))
            out.append(g.normal(0.0, std, fo * fi))
            out.append(g.normal(0.0, bias_std, fo) if bias_std > 0 else np.zeros(fo))
    return np.concatenate(out).astype(np.float32)


@dataclass
class Problem:
    cfg: dict
    res_pts: np.ndarray
    res_counts: np.ndarray
    obs_pts: np.ndarray
    obs_vals: np.ndarray
    obs_counts: np.ndarray
    face_pts: np.ndarray
    face_counts: np.ndarray
    theta0: np.ndarray
    seed: int = 0
    extra: dict = field(default_factory=dict)
    ghost_pts: np.ndarray | None = None
    ghost_counts: np.ndarray | None = None

    @property
    def n_res(self) -> int:
        return int(self.res_counts.sum())


def make_problem(cfg, seed=0, res_counts=None, n_obs=None, n_face=None,
                 bias_std=0.0, noise=None, face_counts=None, obs_counts=None) -> Problem:
    """Sample a full synthetic problem for ``cfg``.

    Collocation and observation points are uniform in each net's interior
    cell; observation values are the analytic velocity plus Gaussian noise of
    ``noise * std_c`` per component, std over that net's observations.  Face
    points are uniform on the shared face: the face's axis coordinate is the
    boundary value, the others are uniform over the lower net's cell.
    """
    di, ds = d_in(cfg), cfg["d_space"]
    nn = n_nets(cfg)
    if res_counts is None:
        res_counts = residual_counts(cfg, seed)
    res_counts = np.asarray(res_counts, np.int64)
    if obs_counts is None:
        n_obs = cfg["n_obs"] if n_obs is None else n_obs
        obs_counts = np.full(nn, int(n_obs), np.int64)
    obs_counts = np.asarray(obs_counts, np.int64)
    noise = cfg["noise"] if noise is None else noise
    fl = faces(cfg)
    if face_counts is None:
        n_face = cfg["n_face"] if n_face is None else n_face
        face_counts = np.full(len(fl), int(n_face), np.int64)
    face_counts = np.asarray(face_counts, np.int64)

    g_res, g_obs, g_noise, g_face = _rng(seed, 2), _rng(seed, 3), _rng(seed, 4), _rng(seed, 6)
    res, obs, obsv = [], [], []
    for k in range(nn):
        lo, hi = net_box(cfg, k)
        res.append(_uniform_in_box(g_res, lo, hi, int(res_counts[k])))
        po = _uniform_in_box(g_obs, lo, hi, int(obs_counts[k]))
        vals = flow_values(cfg, po)[:, :ds] if len(po) else np.zeros((0, ds))
        if len(po) > 1 and noise > 0:
            std = vals.std(axis=0)
            vals = vals + noise * std[None, :] * g_noise.normal(0.0, 1.0, vals.shape)
        obs.append(po)
        obsv.append(vals)
    fpts = []
    for f, (klo, khi, ax) in enumerate(fl):
        lo, hi = net_box(cfg, klo)
        p = _uniform_in_box(g_face, lo, hi, int(face_counts[f]))
        p[:, ax] = hi[ax]
        fpts.append(p)
    cat = lambda xs, w: (np.concatenate(xs) if xs else np.zeros((0, w))).astype(np.float32).reshape(-1, w)
    return Problem(
        cfg=cfg,
        res_pts=cat(res, di), res_counts=res_counts,
        obs_pts=cat(obs, di), obs_vals=cat(obsv, ds), obs_counts=obs_counts,
        face_pts=cat(fpts, di), face_counts=face_counts,
        theta0=init_params(cfg, seed, bias_std), seed=seed,
    )


def cell_fp32(cfg, a, x):
    """Cell index of coordinate(s) x along axis a with the float32 rule of the
    interface (floor((x - lo) * (splits / (hi - lo))), clamped); -1 outside."""
    x = np.asarray(x, np.float32)
    lo, hi = np.float32(cfg["lo"][a]), np.float32(cfg["hi"][a])
    inv_h = np.float32(cfg["splits"][a] / (cfg["hi"][a] - cfg["lo"][a]))
    q = np.float32(np.float32(x - lo) * inv_h)
    c = np.clip(np.floor(q).astype(np.int64), 0, cfg["splits"][a] - 1)
    return np.where((x >= lo) & (x <= hi), c, -1)


def owner_net(cfg, pts):
    """Net whose cell holds each float32 point (-1 outside the domain)."""
    pts = np.asarray(pts, np.float32)
    net = np.zeros(len(pts), np.int64)
    bad = np.zeros(len(pts), bool)
    for a, st in enumerate(strides(cfg)):
        c = cell_fp32(cfg, a, pts[:, a])
        bad |= c < 0
        net += np.maximum(c, 0) * st
    return np.where(bad, -1, net)


def ghost_points(cfg, n_per_net, delta_space, delta_time=None, seed=0):
    """Volumetric ghost sets: for each net, points uniform in its cell grown by
    delta_space (spatial axes) / delta_time (time axis), clipped to the domain,
    outside the net's own cell (float32 ownership).  Returns (pts, counts)."""
    di, ds = d_in(cfg), cfg["d_space"]
    delta_time = delta_space if delta_time is None else delta_time
    g = _rng(seed, 9)
    out, counts = [], []
    for k in range(n_nets(cfg)):
        lo, hi = net_box(cfg, k)
        d = np.array([delta_space if a < ds else delta_time for a in range(di)])
        glo = np.maximum(lo - d, np.array(cfg["lo"][:di], np.float64))
        ghi = np.minimum(hi + d, np.array(cfg["hi"][:di], np.float64))
        got = np.zeros((0, di), np.float32)
        tries = 0
        while len(got) < n_per_net and tries < 1000:
            cand = _uniform_in_box(g, glo, ghi, 4 * n_per_net + 16).astype(np.float32)
            own = owner_net(cfg, cand)
            cand = cand[(own != k) & (own >= 0)]
            got = np.concatenate([got, cand])[:n_per_net]
            tries += 1
        out.append(got)
        counts.append(len(got))
    pts = np.concatenate(out) if out else np.zeros((0, di), np.float32)
    return pts.astype(np.float32), np.asarray(counts, np.int64)


def with_ghost_layers(pb: Problem, n_per_net, delta_space, delta_time=None, seed=0) -> Problem:
    """The same problem with volumetric ghost sets instead of face points."""
    gp, gc = ghost_points(pb.cfg, n_per_net, delta_space, delta_time, seed)
    pb.ghost_pts, pb.ghost_counts = gp, gc
    return pb


def query_points(cfg, n, seed=0, margin=0.0):
    """Uniform space-time query points in the global box (float32 [n][d_in])."""
    g = _rng(seed, 7)
    di = d_in(cfg)
    lo = np.array(cfg["lo"][:di], np.float64)
    hi = np.array(cfg["hi"][:di], np.float64)
    span = hi - lo
    return _uniform_in_box(g, lo + margin * span, hi - margin * span, n).astype(np.float32)


def random_grad(cfg, seed=0, scale=1e-2):
    """A dense synthetic gradient (for testing the optimizer update alone)."""
    g = _rng(seed, 8)
    return (scale * g.normal(0.0, 1.0, n_nets(cfg) * n_params_net(cfg))).astype(np.float32)
