"""Per-step resampling of the collocation points, the gradient-partial memory
budget and the asynchronous point upload, against the oracle.

The device sampler and the oracle's implement the same counter-based streams
independently; the sampled float32 coordinates must agree bit for bit, and a
step on resampled points must match the oracle's step on those points.
"""
import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import free_run_envelope, rel_l2, step_against_oracle
from tests.test_gpu_parity import GRAD_TOL, _gpu, compare_losses, small_case

pytestmark = pytest.mark.gpu

RESIDUAL = 0


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _setup(name="tgv", precision=0):
    Dpinn = _gpu()
    cfg, pb = small_case(name)
    d = Dpinn(dict(cfg, precision=precision))
    d.set_problem(pb)
    rng = np.random.default_rng(4)
    counts = rng.integers(40, 130, d.n_nets)
    counts[1] = 0
    return d, cfg, pb, counts


def test_sampled_points_match_the_oracle_bit_for_bit():
    d, cfg, pb, counts = _setup()
    ora = oracle.Oracle(cfg)
    seed = 123456789
    d.set_resampling(counts, seed)
    n = int(counts.sum())
    d.eval_loss()                                       # t = 0, no update
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), ora.sample(seed, 0, counts))
    d.step(1)                                           # the step of t = 0
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), ora.sample(seed, 0, counts))
    d.step(1)                                           # t = 1
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), ora.sample(seed, 1, counts))
    d.step(3)                                           # t = 2, 3, 4 in one graph sequence
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), ora.sample(seed, 4, counts))
    d.eval_grad()                                       # t = 5
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), ora.sample(seed, 5, counts))


@pytest.mark.parametrize("name,precision", [("tgv", 0), ("beltrami32", 0), ("beltrami32", 1), ("cyl2d_w150", 0)])
def test_losses_and_gradients_on_resampled_points_match_oracle(name, precision):
    d, cfg, pb, counts = _setup(name, precision)
    seed = 99
    d.set_resampling(counts, seed)
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    ora = oracle.Oracle(cfg)
    pts = ora.sample(seed, 0, counts)
    pb0 = dataclasses.replace(pb, res_pts=pts, res_counts=np.asarray(counts, np.int64))
    ora.set_problem(pb0)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    compare_losses(loss, oloss)
    for k in range(ora.n_nets):
        assert rel_l2(g[k], og[k]) <= GRAD_TOL, (k, rel_l2(g[k], og[k]))
    assert np.all(loss[1, 1] == 0)                      # a net that draws no points has no L_PDE


def test_training_steps_on_fresh_points_track_the_oracle():
    d, cfg, pb, counts = _setup()
    seed = 5
    d.set_resampling(counts, seed)
    ora = oracle.Oracle(cfg)
    for s in range(4):
        ora.set_problem(dataclasses.replace(pb, res_pts=ora.sample(seed, s, counts),
                                            res_counts=np.asarray(counts, np.int64)))
        step_against_oracle(d, ora.step)


def test_switching_off_keeps_the_last_points_and_set_points_takes_over():
    d, cfg, pb, counts = _setup()
    n = int(counts.sum())
    d.set_resampling(counts, 7)
    d.step(2)
    last = d.get_points(RESIDUAL, n)
    d.set_resampling(None)
    d.step(2)
    np.testing.assert_array_equal(d.get_points(RESIDUAL, n), last)
    # user points replace the sampler
    d.set_resampling(counts, 7)
    d.set_points(RESIDUAL, np.asarray(pb.res_pts, np.float32), pb.res_counts)
    d.step(1)
    np.testing.assert_array_equal(d.get_points(RESIDUAL, int(pb.res_counts.sum())),
                                  np.asarray(pb.res_pts, np.float32))


def test_partial_budget_changes_the_plan_not_the_gradient():
    d, cfg, pb, counts = _setup("beltrami32")
    d.eval_grad()
    g0, l0 = d.grad(), d.loss()
    d.set_partial_budget(1)          # as few work items as the plan allows
    d.eval_grad()
    g1, l1 = d.grad(), d.loss()
    ora = oracle.Oracle(cfg, pb)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    compare_losses(l1, oloss)
    for k in range(ora.n_nets):
        assert rel_l2(g1[k], og[k]) <= GRAD_TOL
    assert rel_l2(g1, g0) < 1e-6     # the same sums, in another fixed order
    d.set_partial_budget(0)          # back to the default plan
    d.eval_grad()
    np.testing.assert_array_equal(d.grad(), g0)


def test_async_upload_equals_synchronous_upload():
    """Points uploaded asynchronously for the next step give bit-identical
    steps to synchronous uploads (which the parity tests tie to the oracle)."""
    import torch
    Dpinn = _gpu()
    cfg, pb = small_case("tgv")
    rng = np.random.default_rng(8)
    sets = [np.ascontiguousarray(pb.res_pts + rng.normal(scale=1e-3, size=pb.res_pts.shape), np.float32)
            for _ in range(3)]
    a = Dpinn(cfg)
    a.set_problem(pb)
    b = Dpinn(cfg)
    b.set_problem(pb)
    pinned = [torch.from_numpy(x).pin_memory() for x in sets]
    b.set_points_async(RESIDUAL, pinned[0], pb.res_counts)
    for i in range(3):
        a.set_points(RESIDUAL, sets[i], pb.res_counts)
        a.step(1)
        b.step(1)
        if i + 1 < 3:
            b.set_points_async(RESIDUAL, pinned[i + 1], pb.res_counts)
        np.testing.assert_array_equal(a.loss(), b.loss())
    for x, y in zip(a.get_state()[:3], b.get_state()[:3]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(b.get_points(RESIDUAL, int(pb.res_counts.sum())), sets[2])


def test_async_loss_read_equals_synchronous_read():
    """Loss records queued with loss_async while later steps are already
    queued on the same stream equal the synchronous reads step by step."""
    import torch
    Dpinn = _gpu()
    cfg, pb = small_case("tgv")
    a = Dpinn(cfg)
    a.set_problem(pb)
    b = Dpinn(cfg)
    b.set_problem(pb)
    bufs = [torch.full((b.n_nets, 6), -1.0, dtype=torch.float32).pin_memory() for _ in range(3)]
    s = torch.cuda.Stream()
    for i in range(3):
        b.step(1, s)
        b.loss_async(bufs[i], s)
    s.synchronize()
    for i in range(3):
        a.step(1)
        np.testing.assert_array_equal(bufs[i].numpy(), a.loss())
    with pytest.raises(ValueError):
        b.loss_async(np.zeros((b.n_nets, 6)), s)    # float64
