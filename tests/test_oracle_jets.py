"""Pins of the oracle's forward jets (value, first derivatives, Laplacian).

The jet channels are checked against quantities computed by other means:
complex-step differentiation of the plain value forward (first derivatives,
~1e-15), complex-step differentiation of the first-derivative channel
(second derivatives), central second differences of the value forward, and
PyTorch FP64 autograd on the same network (a library routine).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import net_params, random_points_around, rel_l2, tiny

H = 1e-30
KINDS = ["2s", "2u", "3u", "3s"]


@pytest.mark.parametrize("kind", KINDS)
def test_first_derivatives_complex_step(kind):
    cfg = tiny(kind, width=5, depth=3)
    pb = synth.make_problem(cfg, seed=1, res_counts=[1] * synth.n_nets(cfg), bias_std=0.4)
    ora = oracle.Oracle(cfg)
    for k in range(ora.n_nets):
        th = net_params(pb, k)
        x = random_points_around(cfg, k, 7, seed=k)
        Y = ora.forward(k, th, x, jets=True)
        Yv = ora.forward(k, th, x, jets=False)
        np.testing.assert_array_equal(Y[:, :, 0], Yv[:, :, 0])
        for q in range(ora.d_in):
            xi = np.zeros_like(x)
            xi[:, q] = H
            d = ora.forward_complex(k, th, None, x, xi, jets=False).imag[:, :, 0] / H
            assert rel_l2(Y[:, :, 1 + q], d) < 1e-13, (kind, k, q)


@pytest.mark.parametrize("kind", KINDS)
def test_laplacian_complex_step_and_fd(kind):
    cfg = tiny(kind, width=6, depth=3)
    pb = synth.make_problem(cfg, seed=2, res_counts=[1] * synth.n_nets(cfg), bias_std=0.4)
    ora = oracle.Oracle(cfg)
    ds, lap = cfg["d_space"], ora.d_in + 1
    for k in range(ora.n_nets):
        th = net_params(pb, k)
        x = random_points_around(cfg, k, 6, seed=10 + k)
        Y = ora.forward(k, th, x, jets=True)
        cs = np.zeros(Y.shape[:2])
        fd = np.zeros(Y.shape[:2])
        h = 1e-3 * (synth.net_box(cfg, k)[1] - synth.net_box(cfg, k)[0])
        for s in range(ds):
            xi = np.zeros_like(x)
            xi[:, s] = H
            cs += ora.forward_complex(k, th, None, x, xi, jets=True).imag[:, :, 1 + s] / H
            e = np.zeros_like(x)
            e[:, s] = h[s]
            fp = ora.forward(k, th, x + e, jets=False)[:, :, 0]
            fm = ora.forward(k, th, x - e, jets=False)[:, :, 0]
            fd += (fp - 2 * Y[:, :, 0] + fm) / h[s] ** 2
        assert rel_l2(Y[:, :, lap], cs) < 1e-12, (kind, k)
        assert rel_l2(Y[:, :, lap], fd) < 1e-4, (kind, k)


def _torch_net(cfg, th, k):
    shapes = synth.layer_shapes(cfg)
    lo, hi = synth.net_box(cfg, k)
    c = torch.tensor(0.5 * (lo + hi), dtype=torch.float64)
    s = torch.tensor(2.0 / (hi - lo), dtype=torch.float64)
    t = torch.tensor(th, dtype=torch.float64)
    Ws, off = [], 0
    for (o, i) in shapes:
        W = t[off:off + o * i].reshape(o, i); off += o * i
        b = t[off:off + o]; off += o
        Ws.append((W, b))

    def f(x):
        h = (x - c) * s
        for l, (W, b) in enumerate(Ws):
            h = h @ W.T + b
            if l < len(Ws) - 1:
                h = torch.tanh(h)
        return h
    return f


@pytest.mark.parametrize("kind", KINDS)
def test_jets_match_torch_autograd_fp64(kind):
    cfg = tiny(kind, width=7, depth=4)
    pb = synth.make_problem(cfg, seed=3, res_counts=[1] * synth.n_nets(cfg), bias_std=0.5)
    ora = oracle.Oracle(cfg)
    ds = cfg["d_space"]
    for k in range(ora.n_nets):
        th = net_params(pb, k)
        x = random_points_around(cfg, k, 9, seed=20 + k)
        Y = ora.forward(k, th, x, jets=True)
        f = _torch_net(cfg, th, k)
        xt = torch.tensor(x, requires_grad=True)
        y = f(xt)
        for j in range(ora.d_out):
            g = torch.autograd.grad(y[:, j].sum(), xt, create_graph=True)[0]
            lap = sum(torch.autograd.grad(g[:, s].sum(), xt, retain_graph=True)[0][:, s] for s in range(ds))
            np.testing.assert_allclose(Y[:, j, 0], y[:, j].detach().numpy(), rtol=1e-13, atol=1e-14)
            np.testing.assert_allclose(Y[:, j, 1:1 + ora.d_in], g.detach().numpy(), rtol=1e-12, atol=1e-13)
            np.testing.assert_allclose(Y[:, j, ora.d_in + 1], lap.detach().numpy(), rtol=1e-11, atol=1e-12)


def test_first_layer_scaling_uses_net_box():
    """A net whose box is stretched sees derivatives scaled by 2/(hi-lo)."""
    cfg = tiny("2s", width=3, depth=2)
    pb = synth.make_problem(cfg, seed=4, res_counts=[1] * 4, bias_std=0.2)
    ora = oracle.Oracle(cfg)
    th = net_params(pb, 0)
    x = random_points_around(cfg, 0, 3, seed=1)
    Y = ora.forward(0, th, x)
    # Same net on a box twice as large, evaluated at the mapped point, has
    # half the first derivatives.
    cfg2 = dict(cfg)
    lo, hi = synth.net_box(cfg, 0)
    cfg2.update(splits=[1, 1, 1, 1], lo=[lo[0], lo[1], 0, 0], hi=[2 * hi[0] - lo[0], 2 * hi[1] - lo[1], 0, 0])
    ora2 = oracle.Oracle(cfg2)
    x2 = lo + 2 * (x - lo)
    Y2 = ora2.forward(0, th, x2)
    np.testing.assert_allclose(Y2[:, :, 0], Y[:, :, 0], rtol=1e-13)
    np.testing.assert_allclose(Y2[:, :, 1:3], 0.5 * Y[:, :, 1:3], rtol=1e-12)
    np.testing.assert_allclose(Y2[:, :, 3], 0.25 * Y[:, :, 3], rtol=1e-12)
