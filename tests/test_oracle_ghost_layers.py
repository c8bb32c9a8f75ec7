"""Pins of the volumetric ghost layers (Sec. 2.2, thickness delta > 0).

* complex-step gradient of every per-net loss with ghost sets that reach
  face and corner (diagonal) neighbours;
* PyTorch FP64 double backward of the plain form on the same ghost sets;
* the face limit: ghost points pushed a distance eps off each shared face
  into the neighbour reproduce the face-point losses and gradients as
  eps -> 0 (an independent check of routing, targets and face types);
* the master asymmetry holds in ghost mode too.
"""
import numpy as np
import torch

import oracle
from baseline.plain_form import PlainForm
from paper_2602_15883_b300 import synth
from tests.helpers import rel_l2, tiny, tiny_problem

H = 1e-30


def _ghost_case(kind, seed, n=9, delta=0.3, **kw):
    cfg = tiny(kind, width=4, depth=2, **kw)
    pb = tiny_problem(cfg, seed=seed)
    return cfg, synth.with_ghost_layers(pb, n, delta_space=delta, delta_time=0.25, seed=seed)


def test_ghost_sets_reach_diagonal_neighbours():
    cfg, pb = _ghost_case("2u", 61, n=60)
    go = np.concatenate([[0], np.cumsum(pb.ghost_counts)])
    owners = synth.owner_net(cfg, pb.ghost_pts)
    diag = 0
    for k in range(synth.n_nets(cfg)):
        ck = synth.cell_of_net(cfg, k)
        for B in owners[go[k]:go[k + 1]]:
            assert B != k and B >= 0
            cb = synth.cell_of_net(cfg, B)
            diag += sum(1 for a, b in zip(ck, cb) if a != b) > 1
    assert diag > 0


def test_ghost_gradient_complex_step():
    for kind in ("2u", "3u"):
        cfg, pb = _ghost_case(kind, 62)
        ora = oracle.Oracle(cfg, pb)
        th = np.asarray(pb.theta0, np.float64)
        g, loss = ora.grad(th)
        assert np.any(loss[:, 2] > 0) and np.any(loss[:, 4] > 0)
        npar = ora.n_params
        for A in range(ora.n_nets):
            cs = np.zeros(npar)
            for j in range(npar):
                e = np.zeros(npar)
                e[j] = H
                cs[j] = ora.net_loss_complex(th, A, th_im=e)[5].imag / H
            assert rel_l2(g[A], cs) < 1e-12, (kind, A)


def test_ghost_matches_torch_double_backward_fp64():
    cfg, pb = _ghost_case("3u", 63)
    ora = oracle.Oracle(cfg, pb)
    g, loss = ora.grad(np.asarray(pb.theta0, np.float64))
    pf = PlainForm(pb, dtype=torch.float64)
    rec = pf.losses_and_grads().numpy()
    np.testing.assert_allclose(loss[:, :6], rec, rtol=1e-11, atol=1e-14)
    assert np.all(loss[:, 6:] == 0)   # interface jet terms off
    gt = pf.flat(grads=True).numpy().reshape(ora.n_nets, -1)
    for A in range(ora.n_nets):
        assert rel_l2(g[A], gt[A]) < 1e-11


def test_face_limit_of_ghost_layers():
    cfg = tiny("2u", width=5, depth=2)
    pb = tiny_problem(cfg, seed=64, n_face=6)
    ora_f = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    gf, lf = ora_f.grad(th)
    fl = synth.faces(cfg)
    fo = np.concatenate([[0], np.cumsum(pb.face_counts)])
    eps = 1e-5
    per_net = [[] for _ in range(synth.n_nets(cfg))]
    for f, (a, b, ax) in enumerate(fl):
        x = pb.face_pts[fo[f]:fo[f + 1]].astype(np.float64)
        xa = x.copy(); xa[:, ax] += eps      # net a's ghost point, inside b
        xb = x.copy(); xb[:, ax] -= eps      # net b's ghost point, inside a
        per_net[a].append(xa)
        per_net[b].append(xb)
    pts = [np.concatenate(p) if p else np.zeros((0, 3)) for p in per_net]
    pb.ghost_pts = np.concatenate(pts).astype(np.float32)
    pb.ghost_counts = np.array([len(p) for p in pts], np.int64)
    assert np.all(synth.owner_net(cfg, pb.ghost_pts) >= 0)
    ora_g = oracle.Oracle(cfg, pb)
    gg, lg = ora_g.grad(th)
    np.testing.assert_allclose(lg, lf, rtol=2e-3, atol=1e-9)
    for k in range(ora_f.n_nets):
        assert rel_l2(gg[k], gf[k]) < 2e-3


def test_masters_ignore_spatial_ghost_pressure_in_ghost_mode():
    cfg, pb = _ghost_case("2u", 65, n=80, lambda_obs=0.0, lambda_pde=0.0, lambda_gh_u=0.0, lambda_gh_p_time=0.0,
                          lambda_gh_p_space=1.0)
    ora = oracle.Oracle(cfg, pb)
    g, loss = ora.grad(np.asarray(pb.theta0, np.float64))
    for k in range(ora.n_nets):
        if ora.master[k]:
            assert np.all(g[k] == 0.0) and loss[k, 3] > 0
        elif loss[k, 3] > 0:
            assert np.linalg.norm(g[k]) > 0
