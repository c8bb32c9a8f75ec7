"""Pins of the oracle's optional interface terms beyond C0 continuity (the
Remark in Sec. 2.2): residual matching L_gh_r = mean over ghost points of
||r_A - sg(r_B)||^2 and C1 matching L_gh_c1 = mean of
sum_{c,q} (d_q Y_A,c - sg(d_q Y_B,c))^2.

* The hand-written gradient against complex-step differentiation of the
  per-net loss with the neighbour messages held constant (face and volumetric
  ghost modes).
* Two nets that represent the same function have zero residual and C1
  mismatch (and zero velocity mismatch) on their shared face; a perturbation
  makes them non-zero.
* Both terms depend only on derivatives: a constant added to the neighbour's
  pressure output leaves them unchanged.
"""
import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import rel_l2, tiny, tiny_problem

H = 1e-30


def _with_terms(cfg, lam_r=0.6, lam_c1=0.35):
    return dict(cfg, lambda_gh_r=lam_r, lambda_gh_c1=lam_c1)


@pytest.mark.parametrize("kind", ["2s", "2u", "3u"])
def test_interface_gradient_complex_step(kind):
    cfg = _with_terms(tiny(kind, width=4, depth=2))
    pb = tiny_problem(cfg, seed=21, n_res=3, n_obs=2, n_face=3)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    assert np.all(loss[:, 6] > 0) and np.all(loss[:, 7] > 0)
    npar = ora.n_params
    for A in range(ora.n_nets):
        cs = np.zeros(npar)
        for j in range(npar):
            e = np.zeros(npar)
            e[j] = H
            cs[j] = ora.net_loss_complex(th, A, th_im=e)[5].imag / H
        assert rel_l2(g[A], cs) < 1e-12, (kind, A)
        np.testing.assert_allclose(ora.net_loss_complex(th, A).real, loss[A], rtol=1e-12)


def test_interface_gradient_complex_step_ghost_layers():
    cfg = _with_terms(tiny("2u", width=4, depth=2))
    pb = synth.with_ghost_layers(tiny_problem(cfg, seed=22, n_res=2, n_obs=2), 4, delta_space=0.4,
                                 delta_time=0.2, seed=3)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    assert np.all(loss[:, 6] > 0)
    npar = ora.n_params
    for A in range(ora.n_nets):
        cs = np.zeros(npar)
        for j in range(npar):
            e = np.zeros(npar)
            e[j] = H
            cs[j] = ora.net_loss_complex(th, A, th_im=e)[5].imag / H
        assert rel_l2(g[A], cs) < 1e-12, A


def _two_slab_same_function(perturb=0.0):
    """Two time slabs of one spatial cell whose nets compute the same function:
    net 1's first-layer bias absorbs the shift of its time normalisation."""
    cfg = _with_terms(synth.config("tgv", splits=[1, 1, 2, 1], width=6, depth=3, anchor=[1.0, 2.0, 0.0]))
    pb = synth.make_problem(cfg, seed=5, res_counts=[6, 6], obs_counts=[3, 3], face_counts=[7], bias_std=0.4)
    npar = synth.n_params_net(cfg)
    th = np.array(pb.theta0, np.float64)
    W, din = cfg["width"], synth.d_in(cfg)
    t0 = th[:npar].copy()
    t1 = t0.copy()
    W0 = t0[:W * din].reshape(W, din)
    # both slabs have width 0.5: x_hat_t = 4 (t - c); c_1 - c_0 = 0.5, so
    # x_hat_t(slab 0) = x_hat_t(slab 1) + 2
    t1[W * din:W * din + W] = t0[W * din:W * din + W] + 2.0 * W0[:, din - 1]
    t1 += perturb * np.random.default_rng(1).normal(size=npar)
    th[:npar], th[npar:] = t0, t1
    return cfg, pb, th


def test_identical_functions_have_no_interface_mismatch():
    cfg, pb, th = _two_slab_same_function()
    ora = oracle.Oracle(cfg, pb)
    loss = ora.losses(th)
    assert np.all(loss[:, 2] < 1e-26)     # velocity (C0)
    assert np.all(loss[:, 6] < 1e-24)     # residual matching
    assert np.all(loss[:, 7] < 1e-24)     # C1 matching
    cfg, pb, th = _two_slab_same_function(perturb=1e-3)
    loss = ora.losses(th)
    assert np.all(loss[:, 6] > 1e-12) and np.all(loss[:, 7] > 1e-12)


def test_terms_ignore_the_pressure_level():
    cfg = _with_terms(tiny("2u", width=4, depth=2))
    pb = tiny_problem(cfg, seed=23)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    base = ora.losses(th)
    npar = ora.n_params
    th2 = th.copy()
    th2[(ora.n_nets - 1) * npar + npar - 1] += 3.7     # pressure-output bias of the last net
    moved = ora.losses(th2)
    np.testing.assert_allclose(moved[:, 6:], base[:, 6:], rtol=1e-12, atol=1e-15)
    assert not np.allclose(moved[:, 3:5], base[:, 3:5])   # the C0 pressure terms do see it
