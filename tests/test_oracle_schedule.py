"""Pins of the learning-rate step decay (Table B1) and of the communication
interval I_comm of Algorithm 1 in the oracle.

* decay: the oracle's Adam with lr * factor^floor((t-1)/interval) equals
  torch.optim.Adam driven by torch.optim.lr_scheduler.StepLR;
* I_comm: the messages are recomputed at t = 0, I, 2I, ... and reused
  (stale) in between; with I_comm = 1 the cached stepping equals the plain
  step bitwise; multi-step trajectories equal PyTorch FP64 double backward
  of the plain form with the same interval and decay.
"""
import numpy as np
import torch

import oracle
from baseline.plain_form import PlainForm
from tests.helpers import rel_l2, tiny, tiny_problem


def test_step_decay_matches_torch_steplr():
    cfg = tiny("2u", lr=3e-3, lr_decay_factor=0.3, lr_decay_interval=2)
    ora = oracle.Oracle(cfg)
    npar = ora.n_params
    rng = np.random.default_rng(31)
    th = rng.normal(size=ora.n_nets * npar)
    m, v, t = np.zeros_like(th), np.zeros_like(th), 0
    p = torch.tensor(th).requires_grad_(True)
    opt = torch.optim.Adam([p], lr=cfg["lr"], betas=(cfg["beta1"], cfg["beta2"]), eps=cfg["eps"])
    sch = torch.optim.lr_scheduler.StepLR(opt, step_size=2, gamma=0.3)
    for step in range(7):
        g = rng.normal(size=th.size)
        th, m, v, t = ora.adam(th, m, v, t, g)
        p.grad = torch.tensor(g)
        opt.step()
        sch.step()
        np.testing.assert_allclose(th, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_cached_step_with_interval_one_equals_plain_step():
    cfg = tiny("2u", width=4, depth=2)
    pb = tiny_problem(cfg, seed=32)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    z = np.zeros_like(th)
    a = ora.step(th, z, z, 0)
    b = ora.step_cached(th, z, z, 0, {})
    for x, y in zip(a, b):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_messages_refresh_every_interval():
    cfg = tiny("3u", width=4, depth=2, comm_interval=3)
    pb = tiny_problem(cfg, seed=33)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    m, v, t, cache = np.zeros_like(th), np.zeros_like(th), 0, {}
    ths = [th]
    for step in range(5):
        th, m, v, t, _ = ora.step_cached(th, m, v, t, cache)
        ths.append(th)
        # messages in the cache are those of the last refresh (t = 0 or 3)
        ref_t = 3 * ((t - 1) // 3)
        val, anc = ora.exchange(ths[ref_t])
        np.testing.assert_array_equal(cache["val"], val)
        np.testing.assert_array_equal(cache["anc"], anc)


def test_interval_and_decay_trajectory_matches_torch_fp64():
    cfg = tiny("2u", width=5, depth=3, comm_interval=2, lr=5e-3, lr_decay_factor=0.5, lr_decay_interval=2)
    pb = tiny_problem(cfg, seed=34)
    ora = oracle.Oracle(cfg, pb)
    pf = PlainForm(pb, dtype=torch.float64)
    th = np.asarray(pb.theta0, np.float64)
    m, v, t, cache = np.zeros_like(th), np.zeros_like(th), 0, {}
    for step in range(5):
        th, m, v, t, loss = ora.step_cached(th, m, v, t, cache)
        rec = pf.step().numpy()
        np.testing.assert_allclose(loss[:, :6], rec, rtol=1e-10, atol=1e-14)
        assert np.all(loss[:, 6:] == 0)   # interface jet terms off
    assert rel_l2(th, pf.flat().numpy()) < 1e-10
