"""Parity at the full workload sizes, in the launch configuration the
benchmark times (the whole ensemble in one step), on sampled outputs the
oracle can compute one by one: the loss record and gradient of selected nets
(the smallest net and one other), and queries at sampled points.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2, residual_error, residual_term_scale
from tests.test_gpu_parity import GRAD_TOL, LOSS_TOL, _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


@pytest.mark.parametrize("name,precision", [("tgv", 0), ("beltrami32", 0), ("beltrami128", 0),
                                            ("beltrami32", 1), ("beltrami128", 1),
                                            ("cylinder2d", 0), ("cylinder3d", 0)])
def test_full_size_sampled_nets(name, precision):
    """precision 1 = the tensor-core (3xTF32) jet kernel; the cylinder
    workloads (6 x 150 and 8 x 200 sin nets) run the streamed-weight kernel."""
    Dpinn = _gpu()
    import torch
    cfg = synth.config(name)
    pb = synth.make_problem(cfg, seed=0)
    d = Dpinn(dict(cfg, precision=precision))
    d.set_problem(pb)
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(g))
    ora = oracle.Oracle(cfg, pb)
    small = int(np.argmin(pb.res_counts))
    other = int(np.random.default_rng(0).integers(ora.n_nets))
    nets = sorted({small, other, int(np.nonzero(ora.master)[0][0])})
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64), nets=nets)
    for s, k in enumerate(nets):
        for q in range(6):
            if oloss[s, q] == 0:
                assert loss[k, q] == 0
            else:
                assert abs(loss[k, q] - oloss[s, q]) <= LOSS_TOL * abs(oloss[s, q]) + 1e-12, (k, q)
        assert rel_l2(g[k], og[s]) <= GRAD_TOL, (k, rel_l2(g[k], og[s]))
    # queries at sampled points, values and residuals
    pts = synth.query_points(cfg, 512, seed=1)
    out = d.query(torch.from_numpy(pts).cuda(), want_residual=True).cpu().numpy()
    th = np.asarray(pb.theta0, np.float64)
    ref, nets_q, st = ora.query(th, pts, want_res=True)
    assert st == 0
    do = ora.d_out
    assert rel_l2(out[:, :do], ref[:, :do]) <= LOSS_TOL
    scale = residual_term_scale(query_jets(ora, th, pts, nets_q), cfg)
    assert residual_error(out[:, do:], ref[:, do:], scale) <= LOSS_TOL
