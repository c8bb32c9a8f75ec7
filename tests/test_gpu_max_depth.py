"""The deepest networks the library takes (16 hidden layers) on every kernel
family against the FP64 oracle: the register-tiled FFMA kernels (widths 32,
64, 128), the tensor-core kernels (width 128, 3xTF32) and the streamed-weight
kernel (widths 150 and 200, sin).  At this depth the per-layer biases and the
stash take the most shared and global memory (the tensor-core jet kernel
needs 229,648 of the 232,448 bytes of shared memory a block may have), and
the reverse pass runs its longest chain of layers.  Losses, gradients and
queries (values and residuals) are compared at the stated tolerances."""
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2, residual_error, residual_term_scale
from tests.test_gpu_parity import GRAD_TOL, LOSS_TOL, _gpu, compare_losses

pytestmark = pytest.mark.gpu

MAX_DEPTH = 16

CASES = {
    # name: (base workload, overrides)
    "w32_2d_steady": ("kovasznay", dict(width=32, splits=[2, 1, 1, 1])),
    "w64_2d_unsteady": ("tgv", dict(width=64, splits=[2, 1, 1, 1])),
    "w128_3d_unsteady": ("beltrami32", dict(width=128, splits=[1, 1, 1, 2])),
    "w128_3d_unsteady_tf32x3": ("beltrami32", dict(width=128, splits=[2, 1, 1, 1], precision=1)),
    "w150_2d_unsteady_sin": ("tgv", dict(width=150, activation=1, splits=[1, 1, 1, 2])),
    "w200_3d_unsteady_sin": ("beltrami32", dict(width=200, activation=1, splits=[1, 2, 1, 1])),
}


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _case(name):
    base, over = CASES[name]
    cfg = synth.config(base, depth=MAX_DEPTH, **over)
    nn, nf = synth.n_nets(cfg), len(synth.faces(cfg))
    rng = np.random.default_rng(sum(name.encode()))
    pb = synth.make_problem(cfg, seed=5, bias_std=0.1, res_counts=rng.integers(35, 90, nn),
                            obs_counts=rng.integers(10, 30, nn), face_counts=rng.integers(9, 25, nf))
    return cfg, pb


@pytest.mark.parametrize("name", list(CASES))
def test_max_depth_losses_and_gradients_match_oracle(name):
    Dpinn = _gpu()
    cfg, pb = _case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(g))
    ora = oracle.Oracle(cfg, pb)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    compare_losses(loss, oloss)
    for k in range(ora.n_nets):
        assert rel_l2(g[k], og[k]) <= GRAD_TOL, (k, rel_l2(g[k], og[k]))


@pytest.mark.parametrize("name", ["w64_2d_unsteady", "w128_3d_unsteady_tf32x3", "w200_3d_unsteady_sin"])
def test_max_depth_queries_match_oracle(name):
    import torch
    Dpinn = _gpu()
    cfg, pb = _case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
    pts = synth.query_points(cfg, 300, seed=9)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    ref, nets, st = ora.query(th, pts, want_res=True)
    assert st == 0
    do = ora.d_out
    out = d.query(torch.from_numpy(pts).cuda(), want_residual=True).cpu().numpy()
    assert rel_l2(out[:, :do], ref[:, :do]) <= LOSS_TOL
    scale = residual_term_scale(query_jets(ora, th, pts, nets), cfg)
    assert residual_error(out[:, do:], ref[:, do:], scale) <= LOSS_TOL
