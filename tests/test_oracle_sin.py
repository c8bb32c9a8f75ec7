"""Pins of the oracle with the sin activation (the paper's cylinder cases).

sigma = sin: sigma' = cos, sigma'' = -sin, sigma''' = -cos.  Same checks as
for tanh: complex-step first derivatives and Laplacian of the jets, PyTorch
FP64 autograd jets, complex-step gradient of every per-net loss with all
terms active, and PyTorch FP64 double backward of the plain form.
"""
import numpy as np
import pytest
import torch

import oracle
from baseline.plain_form import PlainForm
from paper_2602_15883_b300 import synth
from tests.helpers import net_params, random_points_around, rel_l2, tiny, tiny_problem

H = 1e-30


@pytest.mark.parametrize("kind", ["2u", "3u"])
def test_sin_jets_complex_step_and_autograd(kind):
    cfg = tiny(kind, width=5, depth=3, activation=1)
    pb = synth.make_problem(cfg, seed=41, res_counts=[1] * synth.n_nets(cfg), bias_std=0.4)
    ora = oracle.Oracle(cfg)
    ds = cfg["d_space"]
    for k in range(ora.n_nets):
        th = net_params(pb, k)
        x = random_points_around(cfg, k, 6, seed=50 + k)
        Y = ora.forward(k, th, x)
        lap = np.zeros(Y.shape[:2])
        for q in range(ora.d_in):
            xi = np.zeros_like(x)
            xi[:, q] = H
            d = ora.forward_complex(k, th, None, x, xi, jets=False).imag[:, :, 0] / H
            assert rel_l2(Y[:, :, 1 + q], d) < 1e-13
            if q < ds:
                lap += ora.forward_complex(k, th, None, x, xi, jets=True).imag[:, :, 1 + q] / H
        assert rel_l2(Y[:, :, -1], lap) < 1e-12
        # PyTorch FP64 autograd on the same network
        lo, hi = synth.net_box(cfg, k)
        xt = torch.tensor(x, requires_grad=True)
        h = (xt - torch.tensor(0.5 * (lo + hi))) * torch.tensor(2.0 / (hi - lo))
        t = torch.tensor(th)
        off = 0
        shapes = synth.layer_shapes(cfg)
        for l, (o, i) in enumerate(shapes):
            W = t[off:off + o * i].reshape(o, i); off += o * i
            b = t[off:off + o]; off += o
            h = h @ W.T + b
            if l < len(shapes) - 1:
                h = torch.sin(h)
        for j in range(ora.d_out):
            g = torch.autograd.grad(h[:, j].sum(), xt, retain_graph=True)[0]
            np.testing.assert_allclose(Y[:, j, 1:1 + ora.d_in], g.numpy(), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("kind", ["2u", "3u"])
def test_sin_loss_gradient_complex_step(kind):
    cfg = tiny(kind, width=4, depth=2, activation=1)
    pb = tiny_problem(cfg, seed=42)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    npar = ora.n_params
    for A in range(ora.n_nets):
        cs = np.zeros(npar)
        for j in range(npar):
            e = np.zeros(npar)
            e[j] = H
            cs[j] = ora.net_loss_complex(th, A, th_im=e)[5].imag / H
        assert rel_l2(g[A], cs) < 1e-12, A


def test_sin_matches_torch_double_backward_fp64():
    cfg = tiny("3u", width=6, depth=3, activation=1)
    pb = tiny_problem(cfg, seed=43, n_res=7, n_obs=5, n_face=4)
    ora = oracle.Oracle(cfg, pb)
    g, loss = ora.grad(np.asarray(pb.theta0, np.float64))
    pf = PlainForm(pb, dtype=torch.float64)
    rec = pf.losses_and_grads().numpy()
    np.testing.assert_allclose(loss[:, :6], rec, rtol=1e-11, atol=1e-14)
    assert np.all(loss[:, 6:] == 0)   # interface jet terms off
    gt = pf.flat(grads=True).numpy().reshape(ora.n_nets, -1)
    for A in range(ora.n_nets):
        assert rel_l2(g[A], gt[A]) < 1e-11


def test_sin_and_tanh_differ():
    """Negative control: the activation switch reaches the forward."""
    cfg_t = tiny("2u", width=4, depth=2)
    cfg_s = tiny("2u", width=4, depth=2, activation=1)
    pb = synth.make_problem(cfg_t, seed=44, res_counts=[1] * 4, bias_std=0.3)
    x = random_points_around(cfg_t, 0, 3, seed=1)
    yt = oracle.Oracle(cfg_t).forward(0, net_params(pb, 0), x)
    ys = oracle.Oracle(cfg_s).forward(0, net_params(pb, 0), x)
    assert np.max(np.abs(yt - ys)) > 1e-3
