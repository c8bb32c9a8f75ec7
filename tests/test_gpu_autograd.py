"""The torch.autograd.Function over the hand-written adjoint.

Checked against the FP64 oracle, against PyTorch FP64 double backward of the
plain form (a library routine), and against central finite differences of
the GPU losses themselves (loose: FP32 losses carry ~1e-7 relative noise).
"""
import os

import numpy as np
import pytest

import oracle
from tests.helpers import rel_l2
from tests.test_gpu_parity import GRAD_TOL, LOSS_TOL, _gpu, small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _setup(name):
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300.autograd import EnsembleModule
    cfg, pb = small_case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
    mod = EnsembleModule(d, pb.theta0)
    return torch, cfg, pb, d, mod


@pytest.mark.parametrize("name", ["tgv", "beltrami32"])
def test_forward_and_backward_match_oracle(name):
    torch, cfg, pb, d, mod = _setup(name)
    out = mod()
    assert out.shape == (d.n_nets,) and out.requires_grad
    ora = oracle.Oracle(cfg, pb)
    og, oloss = ora.grad(np.asarray(pb.theta0, np.float64))
    assert rel_l2(out.detach().cpu().numpy(), oloss[:, 5]) <= LOSS_TOL
    w = torch.linspace(0.5, 2.0, d.n_nets, device="cuda")
    (g,) = torch.autograd.grad((out * w).sum(), mod.theta)
    g = g.cpu().numpy().reshape(d.n_nets, -1)
    wn = w.cpu().numpy()
    for k in range(d.n_nets):
        assert rel_l2(g[k], wn[k] * og[k]) <= GRAD_TOL, k


def test_backward_matches_torch_double_backward_fp64():
    torch, cfg, pb, d, mod = _setup("tgv")
    from baseline.plain_form import PlainForm
    out = mod()
    out.sum().backward()
    g = mod.theta.grad.cpu().numpy().reshape(d.n_nets, -1)
    pf = PlainForm(pb, device="cpu", dtype=torch.float64)
    rec = pf.losses_and_grads().numpy()
    gt = pf.flat(grads=True).numpy().reshape(d.n_nets, -1)
    assert rel_l2(out.detach().cpu().numpy(), rec[:, 5]) <= LOSS_TOL
    for k in range(d.n_nets):
        assert rel_l2(g[k], gt[k]) <= GRAD_TOL, k


def test_backward_matches_finite_differences_of_gpu_losses():
    """The gradient of net A's loss with the neighbour messages held constant
    (the method's gradient) against central differences of the GPU losses.
    The messages are frozen with a long communication interval: one step
    caches them at theta_0, then the parameters are reset to theta_0."""
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300.autograd import ensemble_loss
    cfg, pb = small_case("beltrami128")
    cfg = dict(cfg, comm_interval=1000)
    d = Dpinn(cfg)
    d.set_problem(pb)
    d.step(1)                          # t = 1: messages of theta_0 stay cached
    theta = torch.from_numpy(np.asarray(pb.theta0, np.float32)).cuda()
    d.set_params(theta)
    d.eval_grad()
    g = d.grad()
    npar = d.n_params

    def own_loss(th, k):
        return ensemble_loss(th, d)[k].item()

    for k in (0, d.n_nets - 1):
        gk = g[k]
        for j in np.argsort(-np.abs(gk))[:3]:
            h = 2e-3 * max(1.0, abs(float(theta[k * npar + j])))

            def central(hh):
                tp, tm = theta.clone(), theta.clone()
                tp[k * npar + j] += hh
                tm[k * npar + j] -= hh
                return (own_loss(tp, k) - own_loss(tm, k)) / (2 * hh)
            # Richardson extrapolation removes the O(h^2) truncation term
            fd = (4.0 * central(h / 2) - central(h)) / 3.0
            assert abs(fd - gk[j]) <= 1e-2 * abs(gk[j]), (k, j, fd, gk[j])


def test_torch_adam_drives_the_module_like_the_library_step():
    torch, cfg, pb, d, mod = _setup("tgv")
    opt = torch.optim.Adam([mod.theta], lr=cfg["lr"], betas=(cfg["beta1"], cfg["beta2"]), eps=cfg["eps"])
    opt.zero_grad()
    mod().sum().backward()
    opt.step()
    th_torch = mod.theta.detach().cpu().numpy()
    from paper_2602_15883_b300.binding import Dpinn
    d2 = Dpinn(cfg)
    d2.set_problem(pb)
    d2.step(1)
    th_lib = d2.get_state()[0]
    assert rel_l2(th_torch, th_lib) <= 1e-6


def test_autotuned_schedule_keeps_parity(tmp_path, monkeypatch):
    """Every schedule the tuner tries is a valid plan: after tuning the
    gradient still matches the oracle."""
    monkeypatch.setenv("DPINN_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    Dpinn = _gpu()
    from paper_2602_15883_b300 import autotune
    cfg, pb = small_case("beltrami32")
    d = Dpinn(cfg)
    d.set_problem(pb)
    n_val = int(pb.obs_counts.sum() + 2 * pb.face_counts.sum())
    res = autotune.autotune(d, pb.n_res, n_val, reps=2, jet_candidates=(1, 2, 4), val_candidates=(1, 3))
    assert res["trials"] >= 4 and not res["cached"]
    assert d.get_schedule()["jet_tiles"] == res["jet_tiles"]
    again = autotune.autotune(d, pb.n_res, n_val)
    assert again["cached"]
    for sched in ({"jet_tiles": 1, "val_tiles": 1, "order": 1}, {"jet_tiles": 3, "val_tiles": 2, "order": 0}):
        d.set_schedule(**sched)
        d.eval_grad()
        g = d.grad()
        ora = oracle.Oracle(cfg, pb)
        og, _ = ora.grad(np.asarray(pb.theta0, np.float64))
        for k in range(d.n_nets):
            assert rel_l2(g[k], og[k]) <= GRAD_TOL


def test_graph_captured_plain_form_matches_eager():
    """The CUDA-graph-captured plain form (the benchmark's paper-form arm)
    takes the same steps as the eager one."""
    import torch
    _gpu()
    from baseline.plain_form import PlainForm
    cfg, pb = small_case("tgv")
    a = PlainForm(pb, device="cuda", dtype=torch.float32)
    b = PlainForm(pb, device="cuda", dtype=torch.float32).capture()
    for _ in range(3):
        ra = a.step()
        rb = b.replay()
        torch.testing.assert_close(rb, ra, rtol=1e-4, atol=1e-6)
    torch.testing.assert_close(b.flat(), a.flat(), rtol=1e-4, atol=1e-6)
