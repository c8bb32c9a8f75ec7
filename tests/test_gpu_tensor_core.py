"""GPU-vs-oracle parity of the tensor-core (tcgen05, 3xTF32) jet training kernel.

Same tolerances as the FP32 path: losses <= 1e-5 relative (L2 over nets per
term), weight gradients <= 1e-4 relative (L2 per net).  Cases cover every
channel count of width 128 (C = 4: 2-D steady, 5: 2-D unsteady / 3-D steady,
6: 3-D unsteady), both activations, ragged tiles, several layers, and the
volumetric ghost mode.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import free_run_envelope, rel_l2, step_against_oracle
from tests.test_gpu_parity import GRAD_TOL, compare_losses, small_case

pytestmark = pytest.mark.gpu

TF32X3 = 1


def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2602_15883_b300 import build
    build.build()
    from paper_2602_15883_b300.binding import Dpinn
    return Dpinn


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def tc_case(name):
    if name == "steady2d_w128":        # C = 4
        cfg = synth.config("kovasznay", width=128, depth=4)
        return cfg, synth.make_problem(cfg, seed=2, bias_std=0.1, res_counts=[357], obs_counts=[61])
    if name == "steady3d_w128":        # C = 5, several nets and faces
        cfg = synth.config("beltrami32", unsteady=0, width=128, depth=3, splits=[2, 2, 1, 1],
                           anchor=[0.3, -0.6, 0.1])
        rng = np.random.default_rng(5)
        nn, nf = synth.n_nets(cfg), len(synth.faces(cfg))
        pb = synth.make_problem(cfg, seed=4, bias_std=0.1, res_counts=rng.integers(60, 140, nn),
                                obs_counts=rng.integers(20, 40, nn), face_counts=rng.integers(15, 30, nf))
        return cfg, pb
    return small_case(name)


CASES = ["steady2d_w128", "steady3d_w128", "unsteady2d_w128_deep", "beltrami32", "beltrami128",
         "beltrami_sin", "beltrami_ghost"]


def make(Dpinn, cfg, pb, precision=TF32X3):
    d = Dpinn(dict(cfg, precision=precision))
    d.set_problem(pb)
    return d


@pytest.mark.parametrize("name", CASES)
def test_tf32x3_losses_and_gradients_match_oracle(name):
    Dpinn = _gpu()
    cfg, pb = tc_case(name)
    d = make(Dpinn, cfg, pb)
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    ora = oracle.Oracle(cfg, pb)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    compare_losses(loss, oloss)
    for k in range(ora.n_nets):
        assert rel_l2(g[k], og[k]) <= GRAD_TOL, (k, rel_l2(g[k], og[k]))


def test_tf32x3_path_is_the_one_that_runs():
    """The two precisions give different roundings of the same gradient."""
    Dpinn = _gpu()
    cfg, pb = tc_case("beltrami32")
    a, b = make(Dpinn, cfg, pb, 0), make(Dpinn, cfg, pb, TF32X3)
    a.eval_grad()
    b.eval_grad()
    ga, gb = a.grad(), b.grad()
    assert not np.array_equal(ga, gb)
    assert rel_l2(gb, ga) < 1e-5


def test_tf32x3_one_step_matches_oracle():
    Dpinn = _gpu()
    cfg, pb = tc_case("beltrami32")
    d = make(Dpinn, cfg, pb)
    d.step(1)
    loss = d.loss()
    th1 = d.get_state()[0]
    ora = oracle.Oracle(cfg, pb)
    th0 = np.asarray(pb.theta0, np.float64)
    n = th0.size
    og, _ = ora.grad(th0)
    oth, _, _, _, oloss = ora.step(th0, np.zeros(n), np.zeros(n), 0)
    compare_losses(loss, oloss)
    # Adam's first step is -lr g / (|g| + eps): elements whose gradient is at
    # the rounding-noise floor may take the opposite sign (|diff| <= 2 lr);
    # all others take the oracle's step.
    lr = cfg["lr"]
    og = og.reshape(-1)
    diff = np.abs(th1.astype(np.float64) - oth)
    n_small = 0
    for k in range(ora.n_nets):
        sl = slice(k * ora.n_params, (k + 1) * ora.n_params)
        gk = og[sl]
        big = np.abs(gk) > 1e-3 * np.sqrt(np.mean(gk ** 2))
        n_small += int(np.sum(~big))
        assert np.all(diff[sl][big] <= 1e-3 * lr + 1e-6 * np.abs(th0[sl][big])), k
    assert np.all(diff <= 2 * lr * 1.0001 + 1e-6)
    assert np.linalg.norm(diff) <= 2 * lr * np.sqrt(n_small) + 1e-6 * np.linalg.norm(th0)


def test_tf32x3_losses_only_mode_and_determinism():
    Dpinn = _gpu()
    cfg, pb = tc_case("beltrami128")
    d = make(Dpinn, cfg, pb)
    d.eval_grad()
    g1, l1 = d.grad(), d.loss()
    d.eval_loss()
    l2 = d.loss()
    d.eval_grad()
    g3, l3 = d.grad(), d.loss()
    np.testing.assert_array_equal(l1, l2)
    np.testing.assert_array_equal(l1, l3)
    np.testing.assert_array_equal(g1, g3)


def test_tf32x3_multi_step_trajectory_tracks_oracle():
    Dpinn = _gpu()
    cfg, pb = tc_case("steady3d_w128")
    d = make(Dpinn, cfg, pb)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    t = 0
    for _ in range(4):
        step_against_oracle(d, ora.step)
        th, m, v, t = ora.step(th, m, v, t)[:4]
    assert np.max(np.abs(d.get_state()[0] - th)) <= free_run_envelope(cfg, 4)


@pytest.mark.parametrize("name", ["beltrami32", "steady3d_w128", "beltrami_sin"])
@pytest.mark.parametrize("want_res", [False, True])
def test_tf32x3_queries_match_oracle(name, want_res):
    """Queries through the tensor-core value / jet kernels (routing, the
    anchored pressure of Eq. (18) for master cells, residuals)."""
    import torch
    from tests.helpers import query_jets, residual_error, residual_term_scale
    Dpinn = _gpu()
    cfg, pb = tc_case(name)
    d = make(Dpinn, cfg, pb)
    pts = synth.query_points(cfg, 3001, seed=4)
    out = d.query(torch.from_numpy(pts).cuda(), want_residual=want_res).cpu().numpy()
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    ref, nets, st = ora.query(th, pts, want_res=want_res)
    assert st == 0
    do = ora.d_out
    for c in range(do):
        assert rel_l2(out[:, c], ref[:, c]) <= 1e-5, (c, rel_l2(out[:, c], ref[:, c]))
    if want_res:
        scale = residual_term_scale(query_jets(ora, th, pts, nets), cfg)
        assert residual_error(out[:, do:], ref[:, do:], scale) <= 1e-5


def test_tf32x3_anchor_identity():
    import torch
    Dpinn = _gpu()
    cfg, pb = tc_case("beltrami32")
    cfg = dict(cfg, p_ref=-0.75)
    d = make(Dpinn, cfg, pb)
    ts = np.linspace(0.0, 1.0, 41, dtype=np.float32)
    pts = np.zeros((41, 4), np.float32)
    pts[:, :3] = np.asarray(cfg["anchor"][:3], np.float32)
    pts[:, 3] = ts
    for want in (False, True):
        out = d.query(torch.from_numpy(pts).cuda(), want_residual=want).cpu().numpy()
        assert np.all(out[:, 3] == np.float32(-0.75))
