"""Pins of the oracle's hand-written reverse pass, loss assembly and optimiser.

* Vector-Jacobian products of the jet forward and of the residual against
  complex-step differentiation (every parameter, ~1e-13).
* The full per-net gradient of Eq. (16), with every loss term active, masters
  and both interface types present, against complex-step differentiation of
  the per-net loss in which neighbour messages are constants.
* Central finite differences as a second, independent check.
* PyTorch FP64 autograd double backward (a library routine) on the same
  problem: losses and gradients.
* Adam and clipping against torch.optim.Adam / clip_grad_norm_.
"""
import numpy as np
import pytest
import torch

import oracle
from baseline.plain_form import PlainForm
from paper_2602_15883_b300 import synth
from tests.helpers import net_params, random_points_around, rel_l2, tiny, tiny_problem

H = 1e-30
KINDS = ["2s", "2u", "3u", "3s"]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("jets", [True, False])
def test_forward_vjp_complex_step(kind, jets):
    cfg = tiny(kind, width=4, depth=3)
    pb = synth.make_problem(cfg, seed=7, res_counts=[1] * synth.n_nets(cfg), bias_std=0.5)
    ora = oracle.Oracle(cfg)
    rng = np.random.default_rng(8)
    k = ora.n_nets - 1
    th = net_params(pb, k)
    xpt = random_points_around(cfg, k, 1, seed=3)[0]
    nc = ora.C if jets else 1
    Yb = rng.normal(size=(ora.d_out, nc))
    g = ora.forward_vjp(k, th, xpt, Yb, jets=jets)
    cs = np.zeros_like(g)
    for j in range(len(th)):
        e = np.zeros_like(th)
        e[j] = H
        Y = ora.forward_complex(k, th, e, xpt[None], None, jets=jets)[0]
        cs[j] = np.sum(Yb * Y.imag) / H
    assert rel_l2(g, cs) < 1e-13


@pytest.mark.parametrize("kind", ["2s", "2u", "3u"])
def test_residual_vjp_central_differences(kind):
    """The residual is quadratic in the jets, so central differences are exact
    up to rounding."""
    cfg = tiny(kind)
    ora = oracle.Oracle(cfg)
    rng = np.random.default_rng(9)
    Y = rng.normal(size=(ora.d_out, ora.C))
    rb = rng.normal(size=ora.d_space + 1)
    Yb = ora.residual_vjp(Y, rb)
    fd = np.zeros_like(Y)
    h = 1e-3
    for idx in np.ndindex(*Y.shape):
        e = np.zeros_like(Y)
        e[idx] = h
        fd[idx] = np.dot(rb, (ora.residual(Y + e)[0] - ora.residual(Y - e)[0]) / (2 * h))
    np.testing.assert_allclose(Yb, fd, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("kind", KINDS)
def test_loss_gradient_complex_step_all_terms(kind):
    cfg = tiny(kind, width=4, depth=2)
    pb = tiny_problem(cfg, seed=11)
    ora = oracle.Oracle(cfg, pb)
    assert ora.master.sum() >= 1
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    direct = ora.losses(th)
    np.testing.assert_allclose(loss, direct, rtol=1e-13, atol=1e-15)
    npar = ora.n_params
    for A in range(ora.n_nets):
        cs = np.zeros(npar)
        for j in range(npar):
            e = np.zeros(npar)
            e[j] = H
            cs[j] = ora.net_loss_complex(th, A, th_im=e)[5].imag / H
        assert rel_l2(g[A], cs) < 1e-12, (kind, A)
        # the loss of net A at its own real parameters matches the record
        np.testing.assert_allclose(ora.net_loss_complex(th, A).real, direct[A], rtol=1e-13)


def test_loss_gradient_central_differences():
    cfg = tiny("2u", width=5, depth=3)
    pb = tiny_problem(cfg, seed=12)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, _ = ora.grad(th)
    npar = ora.n_params
    rng = np.random.default_rng(0)
    for A in range(ora.n_nets):
        thA = th[A * npar:(A + 1) * npar]
        for j in rng.choice(npar, 10, replace=False):
            h = 1e-5
            e = np.zeros(npar)
            e[j] = h
            fp = ora.net_loss_complex(th, A, thA=thA + e)[5].real
            fm = ora.net_loss_complex(th, A, thA=thA - e)[5].real
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[A, j]) <= 1e-7 * max(1.0, np.abs(g[A]).max()), (A, j, fd, g[A, j])


@pytest.mark.parametrize("kind", KINDS)
def test_matches_torch_double_backward_fp64(kind):
    cfg = tiny(kind, width=6, depth=3)
    pb = tiny_problem(cfg, seed=13, n_res=7, n_obs=5, n_face=4)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    pf = PlainForm(pb, dtype=torch.float64)
    rec = pf.losses_and_grads().numpy()
    np.testing.assert_allclose(loss[:, :6], rec, rtol=1e-11, atol=1e-14)
    assert np.all(loss[:, 6:] == 0)   # interface jet terms off
    gt = pf.flat(grads=True).numpy().reshape(ora.n_nets, -1)
    for A in range(ora.n_nets):
        assert rel_l2(g[A], gt[A]) < 1e-11, (kind, A)


def test_adam_and_clip_match_torch():
    cfg = tiny("2u", width=4, depth=2, clip_norm=0.05, lr=3e-3)
    ora = oracle.Oracle(cfg)
    npar = ora.n_params
    rng = np.random.default_rng(14)
    th = rng.normal(size=ora.n_nets * npar)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t = 0
    ps = [torch.tensor(th[k * npar:(k + 1) * npar]).requires_grad_(True) for k in range(ora.n_nets)]
    opt = torch.optim.Adam(ps, lr=cfg["lr"], betas=(cfg["beta1"], cfg["beta2"]), eps=cfg["eps"])
    for step in range(4):
        g = rng.normal(size=th.size) * (10.0 ** rng.uniform(-3, 1, th.size))
        th, m, v, t = ora.adam(th, m, v, t, g)
        for k, p in enumerate(ps):
            p.grad = torch.tensor(g[k * npar:(k + 1) * npar])
            torch.nn.utils.clip_grad_norm_([p], cfg["clip_norm"])
        opt.step()
        ref = torch.cat([p.detach() for p in ps]).numpy()
        np.testing.assert_allclose(th, ref, rtol=1e-13, atol=1e-15)
    assert t == 4


def test_adam_first_step_closed_form():
    """With m = v = 0, the first update is -lr * g / (|g| + eps)."""
    cfg = tiny("2s", lr=1e-3)
    ora = oracle.Oracle(cfg)
    rng = np.random.default_rng(15)
    n = ora.n_nets * ora.n_params
    th = rng.normal(size=n)
    g = rng.normal(size=n) * 1e-3
    g[:5] = 0.0
    th1, m, v, t = ora.adam(th, np.zeros(n), np.zeros(n), 0, g)
    np.testing.assert_allclose(th1 - th, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-18)
    assert np.all(th1[:5] == th[:5])
