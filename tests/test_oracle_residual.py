"""Pins of the oracle's Navier-Stokes residual operator (Eqs. (7)-(10)).

Fed the *exact* jets of an analytic incompressible Navier-Stokes solution
(derived here symbolically with sympy, independently of the oracle), the
residual must vanish to rounding.  Three flows exercise the steady 2D, the
unsteady 2D and the unsteady 3D forms.  A wrong sign, a dropped term, a wrong
viscosity factor or a transposed index in the convective term makes the
residual non-zero, which the negative controls below confirm.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import net_params, tiny

x, y, z, t = sp.symbols("x y z t", real=True)


def kovasznay_sym(Re):
    lam = Re / 2 - sp.sqrt(Re ** 2 / 4 + 4 * sp.pi ** 2)
    u = 1 - sp.exp(lam * x) * sp.cos(2 * sp.pi * y)
    v = lam / (2 * sp.pi) * sp.exp(lam * x) * sp.sin(2 * sp.pi * y)
    p = sp.Rational(1, 2) * (1 - sp.exp(2 * lam * x))
    return [u, v, p], [x, y], [x, y]


def tgv_sym(nu):
    f = sp.exp(-2 * nu * t)
    u = sp.cos(x) * sp.sin(y) * f
    v = -sp.sin(x) * sp.cos(y) * f
    p = -sp.Rational(1, 4) * (sp.cos(2 * x) + sp.cos(2 * y)) * f ** 2
    return [u, v, p], [x, y, t], [x, y]


def beltrami_sym(nu, a=sp.pi / 4, d=sp.pi / 2):
    F = sp.exp(-nu * d ** 2 * t)
    E = sp.exp
    u = -a * (E(a * x) * sp.sin(a * y + d * z) + E(a * z) * sp.cos(a * x + d * y)) * F
    v = -a * (E(a * y) * sp.sin(a * z + d * x) + E(a * x) * sp.cos(a * y + d * z)) * F
    w = -a * (E(a * z) * sp.sin(a * x + d * y) + E(a * y) * sp.cos(a * z + d * x)) * F
    p = -a ** 2 / 2 * F ** 2 * (E(2 * a * x) + E(2 * a * y) + E(2 * a * z)
                                + 2 * sp.sin(a * x + d * y) * sp.cos(a * z + d * x) * E(a * (y + z))
                                + 2 * sp.sin(a * y + d * z) * sp.cos(a * x + d * y) * E(a * (z + x))
                                + 2 * sp.sin(a * z + d * x) * sp.cos(a * y + d * z) * E(a * (x + y)))
    return [u, v, w, p], [x, y, z, t], [x, y, z]


def exact_jets(fields, inputs, space, pts):
    """[n][d_out][C] jets: value, d/d(each input), spatial Laplacian."""
    C = len(inputs) + 2
    out = np.zeros((len(pts), len(fields), C))
    for j, f in enumerate(fields):
        exprs = [f] + [sp.diff(f, q) for q in inputs] + [sum(sp.diff(f, s, 2) for s in space)]
        for c, e in enumerate(exprs):
            fn = sp.lambdify(inputs, e, "numpy")
            out[:, j, c] = np.broadcast_to(fn(*[pts[:, i] for i in range(len(inputs))]), (len(pts),))
    return out


def term_scale(Y, ds, nu, unsteady):
    """Magnitude of the individual terms of the momentum residual."""
    C = Y.shape[2]
    s = np.zeros((len(Y), ds))
    for j in range(ds):
        s[:, j] = (np.abs(Y[:, j, 1 + ds]) if unsteady else 0) + np.abs(Y[:, ds, 1 + j]) + nu * np.abs(Y[:, j, C - 1])
        for i in range(ds):
            s[:, j] += np.abs(Y[:, i, 0] * Y[:, j, 1 + i])
    return s


CASES = {
    "kovasznay": (lambda: kovasznay_sym(40), dict(d_space=2, unsteady=0, nu=1 / 40), "kovasznay"),
    "tgv": (lambda: tgv_sym(sp.Rational(1, 100)), dict(d_space=2, unsteady=1, nu=0.01), "tgv"),
    "beltrami": (lambda: beltrami_sym(1), dict(d_space=3, unsteady=1, nu=1.0), "beltrami32"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_residual_vanishes_on_exact_solution(name):
    mk, over, base = CASES[name]
    cfg = synth.config(base, **over)
    fields, inputs, space = mk()
    rng = np.random.default_rng(0)
    n = 40
    pts = rng.uniform(-1, 1, (n, len(inputs)))
    Y = exact_jets(fields, inputs, space, pts)
    ora = oracle.Oracle(cfg)
    r = ora.residual(Y)
    scale = term_scale(Y, cfg["d_space"], cfg["nu"], cfg["unsteady"])
    assert np.max(np.abs(r[:, :-1]) / (scale + 1e-300)) < 1e-12, name
    div_scale = sum(np.abs(Y[:, i, 1 + i]) for i in range(cfg["d_space"]))
    assert np.max(np.abs(r[:, -1]) / (div_scale + 1e-300)) < 1e-12


@pytest.mark.parametrize("name", list(CASES))
def test_residual_detects_wrong_viscosity(name):
    """Negative control: the same jets with nu off by 10 % give r != 0."""
    mk, over, base = CASES[name]
    cfg = synth.config(base, **over)
    cfg["nu"] *= 1.1
    fields, inputs, space = mk()
    pts = np.random.default_rng(1).uniform(-1, 1, (20, len(inputs)))
    Y = exact_jets(fields, inputs, space, pts)
    r = oracle.Oracle(cfg).residual(Y)
    scale = term_scale(Y, cfg["d_space"], cfg["nu"], cfg["unsteady"])
    assert np.max(np.abs(r[:, :-1]) / scale) > 1e-4


def test_residual_detects_time_and_transpose_slips():
    """A jet array with the time channel or the convective index permuted
    no longer satisfies the equations."""
    mk, over, base = CASES["beltrami"]
    cfg = synth.config(base, **over)
    fields, inputs, space = mk()
    pts = np.random.default_rng(2).uniform(-1, 1, (20, 4))
    Y = exact_jets(fields, inputs, space, pts)
    ora = oracle.Oracle(cfg)
    Ysw = Y.copy()
    Ysw[:, :, [1, 2]] = Y[:, :, [2, 1]]  # swap d/dx and d/dy
    assert np.max(np.abs(ora.residual(Ysw)[:, :3])) > 1e-3
    Yt = Y.copy()
    Yt[:, :, 4] *= -1  # flip time derivative
    assert np.max(np.abs(ora.residual(Yt)[:, :3])) > 1e-3


def test_residual_matches_paper_component_form_3d():
    """Eqs. (7)-(10) written component by component for random jets."""
    cfg = tiny("3u")
    ora = oracle.Oracle(cfg)
    rng = np.random.default_rng(3)
    Y = rng.normal(size=(11, 4, 6))
    r = ora.residual(Y)
    nu = cfg["nu"]
    u, v, w, p = (Y[:, j, 0] for j in range(4))
    d = lambda j, q: Y[:, j, 1 + q]   # q: 0=x 1=y 2=z 3=t
    lap = lambda j: Y[:, j, 5]
    r1 = d(0, 3) + (u * d(0, 0) + v * d(0, 1) + w * d(0, 2)) + d(3, 0) - nu * lap(0)
    r2 = d(1, 3) + (u * d(1, 0) + v * d(1, 1) + w * d(1, 2)) + d(3, 1) - nu * lap(1)
    r3 = d(2, 3) + (u * d(2, 0) + v * d(2, 1) + w * d(2, 2)) + d(3, 2) - nu * lap(2)
    r4 = d(0, 0) + d(1, 1) + d(2, 2)
    np.testing.assert_allclose(r, np.stack([r1, r2, r3, r4], 1), rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kind", ["2s", "2u", "3u"])
def test_pressure_shift_invariance(kind):
    """Adding a constant to the pressure output bias leaves the residual and
    L_PDE unchanged (NS depend on p only through its gradient, Sec. 2.2)."""
    cfg = tiny(kind, width=5, depth=3, lambda_obs=0.0, lambda_gh_u=0.0, lambda_gh_p_space=0.0,
               lambda_gh_p_time=0.0)
    pb = synth.make_problem(cfg, seed=5, res_counts=[6] * synth.n_nets(cfg),
                            obs_counts=[0] * synth.n_nets(cfg), face_counts=[0] * len(synth.faces(cfg)),
                            bias_std=0.3)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    L0 = ora.losses(th)
    npar = ora.n_params
    th2 = th.copy()
    for k in range(ora.n_nets):
        th2[k * npar + npar - 1] += 3.7   # last bias entry = pressure output bias
    L1 = ora.losses(th2)
    np.testing.assert_array_equal(L0[:, 1], L1[:, 1])
    g, _ = ora.grad(th)
    assert np.all(g[:, npar - 1] == 0.0)
    assert np.all(np.abs(g[:, npar - 2]) > 0)   # last velocity bias is used
