"""Closed-form pins of the data loss (Eq. (3)), the ghost velocity loss
(Eq. (13)) and the ghost pressure loss with the anchor normalisation
(Eqs. (14)-(15)), with the velocity component weights of Sec. 3.3.

With the output-layer weight W_L set to zero every net is the constant map
x -> b_L (its output bias): all derivative channels vanish, so the Navier-
Stokes residuals and L_PDE are exactly zero, the neighbour messages are the
neighbours' biases, and an anchored master pressure p(x, t) - p(x_anc, t) is
exactly zero.  The losses then reduce to short sums that are worked out by
hand below (with the arithmetic written out), and to the same sums over random
multi-net problems with both face types.  A plausible slip in the oracle -
dividing by N * d_s as a mean over components would, weighting the pressure
with a component weight, normalising the own pressure instead of the
neighbour's, or the wrong sign in Eq. (15) - changes these values.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import tiny, tiny_problem


def _constant_nets(cfg, theta, biases):
    """Parameters with W_L = 0 and b_L = biases[k] for every net k."""
    npar = synth.n_params_net(cfg)
    do, W = synth.d_out(cfg), cfg["width"]
    th = np.array(theta, np.float64).reshape(-1, npar)
    th[:, npar - do - do * W: npar - do] = 0.0
    th[:, npar - do:] = biases
    return th.ravel()


def _problem(cfg, res, res_c, obs, obs_v, obs_c, face, face_c, theta):
    f32 = lambda a, w: np.asarray(a, np.float32).reshape(-1, w)
    di, ds = synth.d_in(cfg), cfg["d_space"]
    return SimpleNamespace(cfg=cfg, res_pts=f32(res, di), res_counts=np.asarray(res_c, np.int64),
                           obs_pts=f32(obs, di), obs_vals=f32(obs_v, ds), obs_counts=np.asarray(obs_c, np.int64),
                           face_pts=f32(face, di), face_counts=np.asarray(face_c, np.int64), theta0=theta)


def test_hand_worked_single_net_data_loss():
    """One steady 2-D net, b_L = (0.5, -0.25, 0.75), w = (1, 2.5, 7) (the
    third weight has no velocity component in 2-D and must not enter),
    observations u_obs = (1, 0) and (0, 1):
      L_obs = (1/2) [1 (0.5 - 1)^2 + 2.5 (-0.25 - 0)^2 + 1 (0.5 - 0)^2 + 2.5 (-0.25 - 1)^2]
            = (1/2) [0.25 + 0.15625 + 0.25 + 3.90625] = 2.28125,
    L_PDE = 0 (constant map), no faces; L_total = lambda_obs * 2.28125."""
    cfg = synth.config("kovasznay", comp_w=[1.0, 2.5, 7.0], lambda_obs=1.3, lambda_pde=0.7)
    pb0 = synth.make_problem(cfg, seed=3)
    th = _constant_nets(cfg, pb0.theta0, [[0.5, -0.25, 0.75]])
    pb = _problem(cfg, res=[[0.1, 0.2], [0.7, -0.3], [-0.4, 1.2]], res_c=[3],
                  obs=[[0.2, 0.1], [0.9, 1.4]], obs_v=[[1.0, 0.0], [0.0, 1.0]], obs_c=[2],
                  face=np.zeros((0, 2)), face_c=[], theta=th)
    ora = oracle.Oracle(cfg, pb)
    L = ora.losses(th)[0]
    assert L[0] == pytest.approx(2.28125, rel=1e-14)
    assert L[1] == 0.0
    assert L[2] == L[3] == L[4] == 0.0
    assert L[5] == pytest.approx(1.3 * 2.28125, rel=1e-14)


def test_hand_worked_two_net_ghost_losses():
    """Two steady 2-D nets split along x, anchor in net 0 (net 0 is the
    master), one spatial face with two points; b_0 = (0.5, -0.25, 0.75),
    b_1 = (0.25, 0.5, -1.0), w = (1, 2.5, 7); two observations on net 0 as
    in the single-net case, none on net 1.  N_gh = 2 for both nets.
      L_gh_u (both)   = (1/2) * 2 * [1 (0.5 - 0.25)^2 + 2.5 (-0.25 - 0.5)^2]
                      = 0.0625 + 1.40625 = 1.46875
      L_gh_p^space(0) = (p_0 - p_1)^2 = (0.75 + 1)^2 = 3.0625   (net 1 is not a master: raw p_1;
                                                                 reported, weight 0 on the master)
      L_gh_p^space(1) = (p_1 - (p_0(x) - p_0(x_anc)))^2 = (-1 - 0)^2 = 1   (Eq. (15))
      L_total(0) = l_obs 2.28125 + l_gh_u 1.46875
      L_total(1) = l_gh_u 1.46875 + l_space 1."""
    cfg = synth.config("kovasznay", splits=[2, 1, 1, 1], anchor=[-0.2, 0.3, 0.0], comp_w=[1.0, 2.5, 7.0],
                       lambda_obs=1.3, lambda_pde=0.7, lambda_gh_u=0.45, lambda_gh_p_space=0.8,
                       lambda_gh_p_time=0.55)
    pb0 = synth.make_problem(cfg, seed=4)
    th = _constant_nets(cfg, pb0.theta0, [[0.5, -0.25, 0.75], [0.25, 0.5, -1.0]])
    lo, hi = synth.net_box(cfg, 0)
    xf = hi[0]   # the shared face x = x_f
    pb = _problem(cfg, res=[[-0.3, 0.2], [0.6, 0.5]], res_c=[1, 1],
                  obs=[[-0.4, 0.1], [-0.2, 1.4]], obs_v=[[1.0, 0.0], [0.0, 1.0]], obs_c=[2, 0],
                  face=[[xf, 0.1], [xf, 1.1]], face_c=[2], theta=th)
    ora = oracle.Oracle(cfg, pb)
    assert list(ora.master) == [1, 0]
    L = ora.losses(th)
    assert L[0, 0] == pytest.approx(2.28125, rel=1e-14) and L[1, 0] == 0.0
    assert L[0, 1] == 0.0 and L[1, 1] == 0.0
    assert L[0, 2] == pytest.approx(1.46875, rel=1e-14) and L[1, 2] == pytest.approx(1.46875, rel=1e-14)
    assert L[0, 3] == pytest.approx(3.0625, rel=1e-14) and L[1, 3] == pytest.approx(1.0, rel=1e-14)
    assert L[0, 4] == 0.0 and L[1, 4] == 0.0
    assert L[0, 5] == pytest.approx(1.3 * 2.28125 + 0.45 * 1.46875, rel=1e-14)
    assert L[1, 5] == pytest.approx(0.45 * 1.46875 + 0.8 * 1.0, rel=1e-14)


@pytest.mark.parametrize("kind", ["2s", "2u", "3u"])
def test_constant_nets_random_problems(kind):
    """The same sums over random problems: several nets, several points per
    face and observation set (some empty), both face types, masters on both
    sides of temporal faces, non-uniform component weights."""
    cfg = tiny(kind, comp_w=[0.7, 1.9, 3.1])
    pb = tiny_problem(cfg, seed=8, n_res=4, n_obs=5, n_face=4)
    nn = synth.n_nets(cfg)
    ds, do = cfg["d_space"], synth.d_out(cfg)
    b = np.random.default_rng(5).normal(size=(nn, do))
    th = _constant_nets(cfg, pb.theta0, b)
    pb.theta0 = th
    ora = oracle.Oracle(cfg, pb)
    L = ora.losses(th)
    w = np.array(cfg["comp_w"][:ds])
    # Eq. (3): observations of net k, squared 2-norm weighted per component, / N_obs,k
    off = np.concatenate([[0], np.cumsum(pb.obs_counts)])
    for k in range(nn):
        ov = pb.obs_vals[off[k]:off[k + 1]].astype(np.float64)
        exp = (w * (b[k, :ds] - ov) ** 2).sum() / len(ov) if len(ov) else 0.0
        assert L[k, 0] == pytest.approx(exp, rel=1e-13, abs=0.0)
    assert np.all(L[:, 1] == 0.0)
    # Eqs. (13)-(15): every face point of a net's faces contributes the same
    # constant difference; the neighbour's pressure is anchored when it is a master
    n_gh = np.zeros(nn)
    gu, gs, gt = np.zeros(nn), np.zeros(nn), np.zeros(nn)
    for f, (a, c, ax) in enumerate(synth.faces(cfg)):
        n = pb.face_counts[f]
        is_time = cfg["unsteady"] and ax == cfg["d_space"]
        for own, oth in ((a, c), (c, a)):
            n_gh[own] += n
            gu[own] += n * (w * (b[own, :ds] - b[oth, :ds]) ** 2).sum()
            p_oth = 0.0 if ora.master[oth] else b[oth, ds]
            (gt if is_time else gs)[own] += n * (b[own, ds] - p_oth) ** 2
    for k in range(nn):
        s = 1.0 / n_gh[k] if n_gh[k] else 0.0
        assert L[k, 2] == pytest.approx(gu[k] * s, rel=1e-13, abs=1e-300)
        assert L[k, 3] == pytest.approx(gs[k] * s, rel=1e-13, abs=1e-300)
        assert L[k, 4] == pytest.approx(gt[k] * s, rel=1e-13, abs=1e-300)
        lam_s = 0.0 if ora.master[k] else cfg["lambda_gh_p_space"]
        tot = cfg["lambda_obs"] * L[k, 0] + cfg["lambda_gh_u"] * L[k, 2] + lam_s * L[k, 3] \
            + cfg["lambda_gh_p_time"] * L[k, 4]
        assert L[k, 5] == pytest.approx(tot, rel=1e-13, abs=1e-300)
