"""Invariants the paper states, pinned on the oracle.

* Decomposition layout: boxes, faces, master set (Sec. 2.2, Algorithm 1).
* Spatial asymmetry: a master never receives gradient from the spatial ghost
  pressure term (lambda^space = 0 on masters), while the temporal term stays
  active everywhere (Sec. 2.2 items (1)-(2)).
* With lambda^space = lambda^time the split terms add up to the unsplit
  L_gh_p of Eq. (14).
* Anchor identity: the anchored output pressure of a master cell equals
  p_ref at x_anc for every time (Eq. (15), Eq. (18)).
* With every ghost weight zero, one K x M step equals K*M independent
  single-net steps, bitwise (the nets are independent, Sec. 2.2).
* Query routing: half-open cells, the last one closed, out-of-domain flagged.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import rel_l2, tiny, tiny_problem


@pytest.mark.parametrize("name", ["kovasznay", "tgv", "beltrami32", "beltrami128"])
def test_layout_matches_generator_geometry(name):
    cfg = synth.config(name)
    ora = oracle.Oracle(cfg)
    assert ora.n_nets == synth.n_nets(cfg)
    assert ora.n_params == synth.n_params_net(cfg)
    fl = synth.faces(cfg)
    assert ora.n_faces == len(fl)
    for f, (a, b, ax) in enumerate(fl):
        assert tuple(ora.faces[f, :3]) == (a, b, ax)
        assert ora.faces[f, 3] == (1 if cfg["unsteady"] and ax == cfg["d_space"] else 0)
    for k in range(ora.n_nets):
        lo, hi = synth.net_box(cfg, k)
        np.testing.assert_allclose(ora.box_lo[k, :lo.size], lo, rtol=0, atol=1e-15)
        np.testing.assert_allclose(ora.box_hi[k, :hi.size], hi, rtol=0, atol=1e-15)
    # masters: the nets of the anchor's spatial cell, one per time slab
    ds = cfg["d_space"]
    slabs = cfg["splits"][ds] if cfg["unsteady"] else 1
    assert ora.master.sum() == slabs
    for k in np.nonzero(ora.master)[0]:
        lo, hi = synth.net_box(cfg, k)
        assert all(lo[a] <= cfg["anchor"][a] < hi[a] for a in range(ds))


def test_known_face_counts():
    # 4x4x2 TGV: x faces 3*4*2, y faces 4*3*2, t faces 4*4*1 -> 48 space + 16 time
    ora = oracle.Oracle(synth.config("tgv"))
    assert ora.n_faces == 64 and ora.faces[:, 3].sum() == 16
    ora = oracle.Oracle(synth.config("beltrami32"))
    assert ora.n_faces == 72 and ora.faces[:, 3].sum() == 24
    ora = oracle.Oracle(synth.config("beltrami128"))
    assert ora.n_faces == 352 and ora.faces[:, 3].sum() == 96


@pytest.mark.parametrize("kind", ["2s", "2u", "3u"])
def test_masters_ignore_spatial_ghost_pressure(kind):
    cfg = tiny(kind, lambda_obs=0.0, lambda_pde=0.0, lambda_gh_u=0.0, lambda_gh_p_time=0.0,
               lambda_gh_p_space=1.0)
    pb = tiny_problem(cfg, seed=21)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    g, loss = ora.grad(th)
    has_space_face = np.zeros(ora.n_nets, bool)
    for (a, b, ax, tm) in ora.faces:
        if not tm:
            has_space_face[a] = has_space_face[b] = True
    for k in range(ora.n_nets):
        if ora.master[k]:
            assert np.all(g[k] == 0.0) and loss[k, 5] == 0.0
            if has_space_face[k]:
                assert loss[k, 3] > 0.0   # the term is still reported
        elif has_space_face[k]:
            assert np.linalg.norm(g[k]) > 0


def test_temporal_term_active_on_masters():
    cfg = tiny("2u", lambda_obs=0.0, lambda_pde=0.0, lambda_gh_u=0.0, lambda_gh_p_space=0.0,
               lambda_gh_p_time=1.0)
    pb = tiny_problem(cfg, seed=22)
    ora = oracle.Oracle(cfg, pb)
    g, loss = ora.grad(np.asarray(pb.theta0, np.float64))
    for k in np.nonzero(ora.master)[0]:
        assert loss[k, 4] > 0 and np.linalg.norm(g[k]) > 0


def test_split_terms_sum_to_unsplit_ghost_pressure():
    cfg = tiny("3u", lambda_gh_p_space=0.8, lambda_gh_p_time=0.8)
    pb = tiny_problem(cfg, seed=23, n_face=6)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    rec = ora.losses(th)
    val, anc = ora.exchange(th)
    fo = np.concatenate([[0], np.cumsum(pb.face_counts)])
    for A in range(ora.n_nets):
        num, ngh = 0.0, 0
        for f, (a, b, ax, tm) in enumerate(ora.faces):
            if A not in (a, b):
                continue
            side = 0 if A == a else 1
            other = (a, b)[1 - side]
            for i in range(fo[f], fo[f + 1]):
                P = val[i, 1 - side, -1] - (anc[i, 1 - side] if ora.master[other] else 0.0)
                num += (val[i, side, -1] - P) ** 2
                ngh += 1
        unsplit = num / ngh if ngh else 0.0
        np.testing.assert_allclose(rec[A, 3] + rec[A, 4], unsplit, rtol=1e-12, atol=1e-16)


def test_exchange_values_are_each_sides_own_prediction():
    cfg = tiny("2u", width=5)
    pb = tiny_problem(cfg, seed=24)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    val, anc = ora.exchange(th)
    fo = np.concatenate([[0], np.cumsum(pb.face_counts)])
    npar = ora.n_params
    for f, (a, b, ax, tm) in enumerate(ora.faces):
        x = pb.face_pts[fo[f]:fo[f + 1]].astype(np.float64)
        for side, k in enumerate((a, b)):
            y = ora.forward(k, th[k * npar:(k + 1) * npar], x, jets=False)[:, :, 0]
            np.testing.assert_array_equal(val[fo[f]:fo[f + 1], side], y)
            if ora.master[k]:
                xa = x.copy()
                xa[:, :2] = np.float32(cfg["anchor"][:2])
                pa = ora.forward(k, th[k * npar:(k + 1) * npar], xa, jets=False)[:, -1, 0]
                np.testing.assert_array_equal(anc[fo[f]:fo[f + 1], side], pa)
            else:
                assert np.all(anc[fo[f]:fo[f + 1], side] == 0)


@pytest.mark.parametrize("kind", ["2u", "3u"])
def test_anchor_identity_in_query(kind):
    cfg = tiny(kind, p_ref=0.3125)
    pb = tiny_problem(cfg, seed=25)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    ds = cfg["d_space"]
    ts = np.linspace(cfg["lo"][ds], cfg["hi"][ds], 9)
    pts = np.zeros((len(ts), ds + 1), np.float32)
    pts[:, :ds] = np.float32(cfg["anchor"][:ds])
    pts[:, ds] = ts
    out, nets, st = ora.query(th, pts)
    assert st == 0 and all(ora.master[nets])
    assert np.all(out[:, ds] == 0.3125)


def test_decomposition_equals_independent_nets_without_ghost_terms():
    cfg = tiny("2u", width=5, depth=3, lambda_gh_u=0.0, lambda_gh_p_space=0.0, lambda_gh_p_time=0.0)
    pb = tiny_problem(cfg, seed=26)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    npar = ora.n_params
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    th1, m1, v1, t1, loss = ora.step(th, m, v, 0)
    ro = np.concatenate([[0], np.cumsum(pb.res_counts)])
    oo = np.concatenate([[0], np.cumsum(pb.obs_counts)])
    for k in range(ora.n_nets):
        lo, hi = synth.net_box(cfg, k)
        c1 = dict(cfg)
        c1.update(splits=[1, 1, 1, 1], lo=list(lo) + [0], hi=list(hi) + [0], anchor=list(lo) + [0])
        sub = synth.Problem(
            cfg=c1, res_pts=pb.res_pts[ro[k]:ro[k + 1]], res_counts=np.array([ro[k + 1] - ro[k]]),
            obs_pts=pb.obs_pts[oo[k]:oo[k + 1]], obs_vals=pb.obs_vals[oo[k]:oo[k + 1]],
            obs_counts=np.array([oo[k + 1] - oo[k]]), face_pts=np.zeros((0, 3), np.float32),
            face_counts=np.zeros(0, np.int64), theta0=pb.theta0[k * npar:(k + 1) * npar])
        o1 = oracle.Oracle(c1, sub)
        thk = th[k * npar:(k + 1) * npar]
        a, _, _, _, l1 = o1.step(thk, np.zeros(npar), np.zeros(npar), 0)
        np.testing.assert_array_equal(a, th1[k * npar:(k + 1) * npar])
        # ghost terms are still reported by the decomposed run; they carry no weight
        np.testing.assert_array_equal(l1[0][[0, 1, 5]], loss[k][[0, 1, 5]])


def test_query_routing_half_open_cells():
    cfg = tiny("2s")   # [-0.5, 1] x [-0.5, 1.5] split 2 x 2
    pb = tiny_problem(cfg, seed=27)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    pts = np.array([[-0.5, -0.5], [0.25, 0.5], [0.2499, 0.4999], [1.0, 1.5], [0.9, -0.4],
                    [1.01, 0.0], [0.0, -0.6]], np.float32)
    out, nets, st = ora.query(th, pts)
    assert list(nets[:5]) == [0, 3, 0, 3, 1]
    assert list(nets[5:]) == [-1, -1] and st == -1
    # each routed point's output is its own net's prediction
    npar = ora.n_params
    for i in range(5):
        k = nets[i]
        y = ora.forward(k, th[k * npar:(k + 1) * npar], pts[i:i + 1].astype(np.float64), jets=False)[0, :, 0]
        p = y[2]
        if ora.master[k]:
            xa = np.array([cfg["anchor"][:2]], np.float32).astype(np.float64)
            p = p - ora.forward(k, th[k * npar:(k + 1) * npar], xa, jets=False)[0, -1, 0]
        np.testing.assert_array_equal(out[i, :2], y[:2])
        assert out[i, 2] == p + cfg["p_ref"]


def test_query_residual_equals_residual_of_jets():
    cfg = tiny("3u", width=5)
    pb = tiny_problem(cfg, seed=28)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    pts = synth.query_points(cfg, 17, seed=3, margin=0.01)
    out, nets, st = ora.query(th, pts, want_res=True)
    npar = ora.n_params
    for i in range(len(pts)):
        k = nets[i]
        Y = ora.forward(k, th[k * npar:(k + 1) * npar], pts[i:i + 1].astype(np.float64))
        np.testing.assert_array_equal(out[i, 4:], ora.residual(Y)[0])


def test_threaded_gradient_is_deterministic_and_matches_serial():
    cfg = tiny("2u", width=6)
    pb = tiny_problem(cfg, seed=29, n_res=40, n_obs=20, n_face=10)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    oracle.set_threads(1)
    g1, l1 = ora.grad(th)
    oracle.set_threads(4)
    g4, l4 = ora.grad(th)
    g4b, _ = ora.grad(th)
    oracle.set_threads(1)
    np.testing.assert_array_equal(g4, g4b)
    assert rel_l2(g4, g1) < 1e-14
