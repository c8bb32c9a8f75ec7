"""Edge cases of the streamed-weight kernel (widths 129-224) against the FP64
oracle: the smallest and largest widths it takes and an exact padded width,
no hidden W x W layer (depth 1), nets without residual or observation
points, ragged tiles, steady and unsteady, tanh and sin; then queries."""
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2, residual_error, residual_term_scale
from tests.test_gpu_parity import GRAD_TOL, _gpu, compare_losses

pytestmark = pytest.mark.gpu

CASES = {
    # name: (base workload, overrides)
    "w129_2d_unsteady_d2": ("tgv", dict(width=129, depth=2, splits=[2, 1, 2, 1], anchor=[1.0, 2.0, 0.0])),
    "w160_3d_steady_d1_sin": ("beltrami32", dict(width=160, depth=1, unsteady=0, activation=1,
                                                   splits=[2, 1, 1, 1], anchor=[-0.5, 0.2, 0.1])),
    "w224_2d_steady_d3": ("kovasznay", dict(width=224, depth=3, splits=[2, 2, 1, 1])),
    "w224_3d_unsteady_d2_sin": ("beltrami32", dict(width=224, depth=2, activation=1, splits=[1, 2, 1, 2],
                                                     anchor=[0.3, -0.4, 0.2])),
}


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _case(name, empty=False):
    base, over = CASES[name]
    cfg = synth.config(base, **over)
    nn, nf = synth.n_nets(cfg), len(synth.faces(cfg))
    rng = np.random.default_rng(sum(name.encode()))
    res = rng.integers(40, 110, nn)
    obs = rng.integers(10, 40, nn)
    if empty:   # one net without residual points, another without observations
        res[0] = 0
        obs[-1] = 0
    pb = synth.make_problem(cfg, seed=2, bias_std=0.1, res_counts=res, obs_counts=obs,
                            face_counts=rng.integers(9, 30, nf))
    return cfg, pb


@pytest.mark.parametrize("empty", [False, True])
@pytest.mark.parametrize("name", list(CASES))
def test_wide_losses_and_gradients_match_oracle(name, empty):
    Dpinn = _gpu()
    cfg, pb = _case(name, empty)
    d = Dpinn(cfg)
    d.set_problem(pb)
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    ora = oracle.Oracle(cfg, pb)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    compare_losses(loss, oloss)
    for k in range(ora.n_nets):
        assert rel_l2(g[k], og[k]) <= GRAD_TOL, (k, rel_l2(g[k], og[k]))
    if empty:
        assert loss[0, 1] == 0 and loss[-1, 0] == 0


@pytest.mark.parametrize("name", ["w129_2d_unsteady_d2", "w224_3d_unsteady_d2_sin"])
def test_wide_queries_match_oracle(name):
    import torch
    Dpinn = _gpu()
    cfg, pb = _case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
    pts = synth.query_points(cfg, 777, seed=8)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    do = ora.d_out
    for want_res in (False, True):
        out = d.query(torch.from_numpy(pts).cuda(), want_residual=want_res).cpu().numpy()
        ref, nets, st = ora.query(th, pts, want_res=want_res)
        assert st == 0
        for c in range(do):
            assert rel_l2(out[:, c], ref[:, c]) <= 1e-5, (c, rel_l2(out[:, c], ref[:, c]))
        if want_res:
            scale = residual_term_scale(query_jets(ora, th, pts, nets), cfg)
            assert residual_error(out[:, do:], ref[:, do:], scale) <= 1e-5
