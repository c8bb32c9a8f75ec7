"""Small configurations and helpers shared by the tests."""
from __future__ import annotations

import math

import numpy as np

from paper_2602_15883_b300 import synth


def tiny(kind: str, width=4, depth=2, **kw) -> dict:
    """Tiny multi-net configurations for exhaustive derivative checks."""
    if kind == "2s":      # steady 2D, 2 x 2 nets
        cfg = synth.config("kovasznay", splits=[2, 2, 1, 1], lo=[-0.5, -0.5, 0, 0], hi=[1.0, 1.5, 0, 0],
                           anchor=[0.1, 0.2, 0.0])
    elif kind == "2u":    # unsteady 2D, 2 x 1 x 2 nets
        cfg = synth.config("tgv", splits=[2, 1, 2, 1], anchor=[1.0, 2.0, 0.0])
    elif kind == "3u":    # unsteady 3D, 1 x 2 x 1 x 2 nets
        cfg = synth.config("beltrami32", splits=[1, 2, 1, 2], anchor=[0.3, -0.4, 0.2])
    elif kind == "3s":    # steady 3D (d_in = 3 without time), 2 x 1 x 1 nets
        cfg = synth.config("beltrami32", unsteady=0, splits=[2, 1, 1, 1], anchor=[-0.2, 0.1, 0.3])
    else:
        raise ValueError(kind)
    cfg.update(width=width, depth=depth, nu=0.37, lambda_obs=1.3, lambda_pde=0.7, lambda_gh_u=0.45,
               lambda_gh_p_space=0.8, lambda_gh_p_time=0.55, comp_w=[1.0, 2.5, 0.6])
    cfg.update(kw)
    return cfg


def tiny_problem(cfg, seed=0, n_res=5, n_obs=4, n_face=3, bias_std=0.3):
    nn = synth.n_nets(cfg)
    nf = len(synth.faces(cfg))
    rng = np.random.default_rng(seed + 100)
    res = rng.integers(max(n_res - 2, 0), n_res + 3, nn)
    obs = rng.integers(max(n_obs - 2, 0), n_obs + 3, nn)
    fc = rng.integers(max(n_face - 1, 0), n_face + 2, nf)
    return synth.make_problem(cfg, seed=seed, res_counts=res, obs_counts=obs, face_counts=fc,
                              bias_std=bias_std)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d


def net_params(pb, k):
    npar = synth.n_params_net(pb.cfg)
    return np.asarray(pb.theta0[k * npar:(k + 1) * npar], np.float64)


def random_points_around(cfg, k, n, seed=0, pad=0.2):
    """Points in net k's box enlarged by ``pad`` of its size (outside allowed)."""
    lo, hi = synth.net_box(cfg, k)
    rng = np.random.default_rng(seed)
    span = hi - lo
    return lo - pad * span + (1 + 2 * pad) * span * rng.uniform(size=(n, lo.size))


def residual_term_scale(Y, cfg):
    """Per point and equation, the sum of magnitudes of the terms of the
    residual, from jets Y [n][d_out][C] (channels: value, d/dx_q, Laplacian)."""
    ds, unst, nu = cfg["d_space"], cfg["unsteady"], cfg["nu"]
    C = Y.shape[2]
    s = np.zeros((len(Y), ds + 1))
    for j in range(ds):
        s[:, j] = np.abs(Y[:, ds, 1 + j]) + nu * np.abs(Y[:, j, C - 1])
        if unst:
            s[:, j] += np.abs(Y[:, j, 1 + ds])
        for i in range(ds):
            s[:, j] += np.abs(Y[:, i, 0] * Y[:, j, 1 + i])
    s[:, ds] = sum(np.abs(Y[:, i, 1 + i]) for i in range(ds))
    return s


def residual_error(gpu_r, ref_r, scale):
    """L2 error of residuals relative to the L2 norm of their term magnitudes."""
    return np.linalg.norm((np.asarray(gpu_r, np.float64) - ref_r).ravel()) / np.linalg.norm(scale.ravel())


def query_jets(ora, th, pts, nets):
    """Oracle jets [n][d_out][C] at routed query points."""
    npar = ora.n_params
    out = np.zeros((len(pts), ora.d_out, ora.C))
    for k in np.unique(nets):
        sel = nets == k
        out[sel] = ora.forward(int(k), th[k * npar:(k + 1) * npar], pts[sel].astype(np.float64))
    return out


def adam_step_bound(beta1, beta2, t):
    """Largest |m_hat_t| / sqrt(v_hat_t) of Adam over all gradient histories
    of length t (Cauchy-Schwarz on the two exponentially weighted sums):
    sqrt(sum_k a_k^2 / b_k) with a_k, b_k the bias-corrected weights of g_k in
    m_hat and of g_k^2 in v_hat.  One Adam update moves an element by at most
    lr times this, whatever its gradients."""
    k = np.arange(1, t + 1)
    a = (1 - beta1) * beta1 ** (t - k) / (1 - beta1 ** t)
    b = (1 - beta2) * beta2 ** (t - k) / (1 - beta2 ** t)
    return float(np.sqrt(np.sum(a * a / b)))


def free_run_envelope(cfg, steps):
    """Bound on |theta_gpu - theta_oracle| per element after `steps` steps
    of two independently integrated trajectories from the same start: each
    step moves each side by at most lr * adam_step_bound (decayed lr is
    smaller), so the two can differ by at most twice the sum.  Elements whose
    gradient lies within FP32 rounding of zero can take such steps with
    opposite signs on the two sides; this is the envelope, not an error."""
    b1, b2, lr = cfg.get("beta1", 0.9), cfg.get("beta2", 0.999), cfg.get("lr", 1e-3)
    return 2.0 * lr * sum(adam_step_bound(b1, b2, t) for t in range(1, steps + 1)) * 1.0001 + 1e-6


def step_against_oracle(d, ora_step, loss_tol=1e-5, param_tol=1e-5):
    """One training step on the GPU handle `d`, compared with the oracle's
    step taken from the GPU's own pre-step state (parameters, Adam moments,
    step count): the loss record at `loss_tol` per term (relative L2 over
    nets) and the parameters after the update at `param_tol` (relative L2).
    `ora_step(th, m, v, t)` returns (th, m, v, t, loss) as Oracle.step does.
    Returns the GPU loss record."""
    th, m, v, t = d.get_state()
    d.step(1)
    loss = d.loss()
    th1, _, _, t1 = d.get_state()
    oth, _, _, ot, oloss = ora_step(th.astype(np.float64), m.astype(np.float64), v.astype(np.float64), t)
    assert t1 == ot == t + 1
    for q in range(6):
        r = oloss[:, q]
        if np.linalg.norm(r) == 0:
            assert np.all(loss[:, q] == 0), q
        else:
            assert rel_l2(loss[:, q], r) <= loss_tol, (t, q, rel_l2(loss[:, q], r))
    assert rel_l2(th1, oth) <= param_tol, (t, rel_l2(th1, oth))
    return loss
