"""GPU-vs-oracle parity of the forward jets themselves (C ABI dpinn_query_jets).

The residuals of Eqs. (7)-(10) are assembled from each net's output jets:
value, first derivative along every input and spatial Laplacian, carried
through the network of Eq. (2).  The other tests see the jets only folded
into residuals, losses and gradients; here every channel of every output is
compared with the FP64 oracle's forward recursion (``ora_forward``) at routed
points, per (output, channel) in relative L2 over the points, with the
1e-5 bar that the method's values, jets and losses must meet.  Routing is
decided in float32 on both sides, so both evaluate the same net per point.

Cases cover every kernel family: register-tiled FP32 at widths 32, 64 and
128, the tcgen05 3xTF32 kernel at width 128, the streamed-weight kernel at
the cylinder widths 150 and 200 (sin), steady and unsteady, 2-D and 3-D, and
the Taylor-Green case at nu = 0.01, whose Laplacian channel carries only
about 1 % of the momentum residual's term magnitude and is therefore poorly
constrained by a residual comparison alone.
"""
import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2
from tests.test_gpu_parity import _gpu, small_case

pytestmark = pytest.mark.gpu

JET_TOL = 1e-5

CASES = [
    ("kovasznay", 0),        # W = 32, steady 2-D
    ("tgv", 0),              # W = 64, nu = 0.01
    ("unsteady3d_w32", 0),   # W = 32, unsteady 3-D
    ("unsteady3d_w64", 0),   # W = 64, unsteady 3-D
    ("beltrami32", 0),       # W = 128 FP32
    ("beltrami32", 1),       # W = 128 tcgen05 3xTF32
    ("beltrami128", 1),
    ("tgv_sin", 0),
    ("cyl2d_w150", 0),       # streamed-weight kernel, padded width 160
    ("cyl3d_w200", 0),       # streamed-weight kernel, padded width 224
]


def _compare(name, precision, n=3001, seed=11):
    Dpinn = _gpu()
    import torch
    cfg, pb = small_case(name)
    cfg = dict(cfg, precision=precision)
    d = Dpinn(cfg)
    d.set_problem(pb)
    pts = synth.query_points(cfg, n, seed=seed)
    got = d.query_jets(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    _, nets, st = ora.query(th, pts)
    assert st == 0
    ref = query_jets(ora, th, pts, nets)
    assert got.shape == ref.shape == (n, ora.d_out, ora.C)
    assert np.all(np.isfinite(got))
    worst = 0.0
    for j in range(ora.d_out):
        for c in range(ora.C):
            e = rel_l2(got[:, j, c], ref[:, j, c])
            worst = max(worst, e)
            assert e <= JET_TOL, (name, precision, j, c, e)
    return worst


@pytest.mark.parametrize("name,precision", CASES)
def test_output_jets_match_oracle_per_channel(name, precision):
    _compare(name, precision)


def test_jets_agree_with_query_values_and_residuals():
    """The jets rows and the regular query rows come from the same forward
    pass: values equal (pressure up to the anchoring of Eq. (18)), and the
    residual assembled on the host from the jets equals the kernel's."""
    Dpinn = _gpu()
    import torch
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    pts = torch.from_numpy(synth.query_points(cfg, 2000, seed=3)).cuda()
    Y = d.query_jets(pts).cpu().numpy().astype(np.float64)
    q = d.query(pts, want_residual=True).cpu().numpy().astype(np.float64)
    ds = cfg["d_space"]
    assert np.array_equal(q[:, :ds], Y[:, :ds, 0])
    # steady-free Eq. (7)-(8) assembled from the jets (unsteady: d_t u_j)
    C = Y.shape[2]
    for j in range(ds):
        r = Y[:, j, 1 + ds] + sum(Y[:, i, 0] * Y[:, j, 1 + i] for i in range(ds)) + Y[:, ds, 1 + j] \
            - cfg["nu"] * Y[:, j, C - 1]
        assert np.max(np.abs(r - q[:, ds + 1 + j])) <= 1e-5 * (1 + np.max(np.abs(r)))
    div = sum(Y[:, i, 1 + i] for i in range(ds))
    assert np.max(np.abs(div - q[:, 2 * ds + 1])) <= 1e-5 * (1 + np.max(np.abs(div)))


def test_empty_jets_query_is_a_no_op():
    Dpinn = _gpu()
    import torch
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    out = d.query_jets(torch.zeros((0, 3), device="cuda"))
    assert out.shape == (0, 3, 5)
