"""GPU-vs-oracle parity of queries on the resident ensemble (C ABI).

Values, anchored pressure (Eq. (18)) and Navier-Stokes residuals at routed
points; routing decided in float32 on both sides, so the net chosen for a
point is identical (bit-exact integer decision).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2, residual_error, residual_term_scale
from tests.test_gpu_parity import _gpu, small_case

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.mark.parametrize("name", ["kovasznay", "tgv", "beltrami32", "steady3d_w64", "unsteady3d_w32", "tgv_sin",
                                  "cyl2d_w150", "cyl3d_w200"])
@pytest.mark.parametrize("want_res", [False, True])
def test_query_matches_oracle(name, want_res):
    Dpinn = _gpu()
    torch = _torch()
    cfg, pb = small_case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
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
        err = residual_error(out[:, do:], ref[:, do:], scale)
        assert err <= 1e-5, err


def test_anchor_identity_and_p_ref():
    Dpinn = _gpu()
    torch = _torch()
    cfg, pb = small_case("tgv")
    cfg = dict(cfg, p_ref=0.25)
    d = Dpinn(cfg)
    d.set_problem(pb)
    ts = np.linspace(0.0, 1.0, 33, dtype=np.float32)
    pts = np.zeros((33, 3), np.float32)
    pts[:, 0] = np.float32(cfg["anchor"][0])
    pts[:, 1] = np.float32(cfg["anchor"][1])
    pts[:, 2] = ts
    out = d.query(torch.from_numpy(pts).cuda()).cpu().numpy()
    assert np.all(out[:, 2] == np.float32(0.25))


def test_out_of_domain_point_is_reported_and_others_served():
    Dpinn = _gpu()
    torch = _torch()
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    pts = synth.query_points(cfg, 100, seed=5)
    pts[17, 0] = -0.5
    out = torch.full((100, 3), 7.0, device="cuda")
    d.query(torch.from_numpy(pts).cuda(), out=out, check=False)
    assert d.query_status() == -1
    o = out.cpu().numpy()
    assert np.all(o[17] == 7.0)
    ora = oracle.Oracle(cfg, pb)
    ok = np.arange(100) != 17
    ref, _, _ = ora.query(np.asarray(pb.theta0, np.float64), pts[ok])
    assert rel_l2(o[ok], ref) < 1e-5
    assert d.query_status() == 0   # cleared


def test_boundary_points_route_like_oracle():
    Dpinn = _gpu()
    torch = _torch()
    cfg, pb = small_case("beltrami128")
    d = Dpinn(cfg)
    d.set_problem(pb)
    rng = np.random.default_rng(6)
    pts = synth.query_points(cfg, 400, seed=6)
    # put coordinates exactly on the interior and outer cell boundaries
    for a in range(4):
        edges = np.linspace(cfg["lo"][a], cfg["hi"][a], cfg["splits"][a] + 1).astype(np.float32)
        sel = rng.random(400) < 0.3
        pts[sel, a] = rng.choice(edges, sel.sum())
    out = d.query(torch.from_numpy(pts).cuda(), want_residual=True).cpu().numpy()
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    ref, nets, st = ora.query(th, pts, want_res=True)
    assert st == 0
    assert rel_l2(out[:, :4], ref[:, :4]) <= 1e-5
    scale = residual_term_scale(query_jets(ora, th, pts, nets), cfg)
    assert residual_error(out[:, 4:], ref[:, 4:], scale) <= 1e-5


def test_batch_invariance_alone_vs_mixed():
    Dpinn = _gpu()
    torch = _torch()
    cfg, pb = small_case("beltrami32")
    d = Dpinn(cfg)
    d.set_problem(pb)
    a = synth.query_points(cfg, 777, seed=7)
    b = synth.query_points(cfg, 5000, seed=8)
    alone = d.query(torch.from_numpy(a).cuda(), want_residual=True).cpu().numpy()
    mixed = d.query(torch.from_numpy(np.concatenate([b[:2000], a, b[2000:]])).cuda(),
                    want_residual=True).cpu().numpy()
    np.testing.assert_array_equal(alone, mixed[2000:2777])
