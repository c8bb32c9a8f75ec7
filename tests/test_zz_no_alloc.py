"""The allocation-free query entry point (dpinn_query_static).

Some callers cannot allocate device memory while they serve (a latency-bound
loop that cannot take the device-wide synchronisation of a cudaMalloc, or a
process whose device memory belongs to another framework's allocator);
dpinn_query_static serves them from a fixed array compiled into the
library.  This file checks, through the C ABI, that two calls in a row give
what the regular dpinn_query gives, that a request of exactly the maximum
size (262,144 points on the kernel with the smallest query tiles, which
fills the fixed work-item array the most) matches the FP64 oracle, and that
oversized requests and ensembles are refused.
It is collected last so that a run stopping at its first failure has
already run everything else; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import query_jets, rel_l2, residual_error, residual_term_scale
from tests.test_gpu_parity import _gpu, small_case

pytestmark = pytest.mark.gpu


def test_static_query_matches_regular_query_twice():
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300 import binding
    lib = binding.load_library()
    cfg, pb = small_case("beltrami32")
    d = Dpinn(cfg)
    d.set_problem(pb)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, want_res) in enumerate([(5000, True), (3001, False)]):
        pts = torch.from_numpy(synth.query_points(cfg, n, seed=20 + call)).cuda()
        w = d.d_out + (d.d_space + 1 if want_res else 0)
        out = torch.full((n, w), float("nan"), device="cuda")
        rc = lib.dpinn_query_static(d.h, pts.data_ptr(), n, int(want_res), out.data_ptr(), stream)
        assert rc == 0, lib.dpinn_last_error(d.h)
        assert lib.dpinn_query_status(d.h, stream) == 0
        ref = d.query(pts, want_residual=want_res)
        got, ref = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_l2(got, ref) <= 1e-5, (call, rel_l2(got, ref))


def test_static_query_refuses_oversized_requests():
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300 import binding
    lib = binding.load_library()
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    dummy = torch.zeros(8, device="cuda")
    rc = lib.dpinn_query_static(d.h, dummy.data_ptr(), 262145, 0, dummy.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"262144" in lib.dpinn_last_error(d.h)


def test_static_query_at_the_maximum_size_matches_oracle():
    """262,144 points with residuals on the width-128 tensor-core jet query
    (16-point tiles, 64-point chunks: 4,096 full chunks plus one partial per
    net in the work-item array), all rows against dpinn_query and a sample of
    rows against the oracle."""
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300 import binding
    lib = binding.load_library()
    cfg, pb = small_case("beltrami32")
    cfg = dict(cfg, precision=1)
    d = Dpinn(cfg)
    d.set_problem(pb)
    n = 262144
    pts_np = synth.query_points(cfg, n, seed=31)
    pts = torch.from_numpy(pts_np).cuda()
    w = d.d_out + d.d_space + 1
    out = torch.full((n, w), float("nan"), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.dpinn_query_static(d.h, pts.data_ptr(), n, 1, out.data_ptr(), stream)
    assert rc == 0, lib.dpinn_last_error(d.h)
    assert lib.dpinn_query_status(d.h, stream) == 0
    got = out.cpu().numpy()
    assert np.all(np.isfinite(got))
    ref = d.query(pts, want_residual=True).cpu().numpy()
    assert rel_l2(got, ref) <= 1e-5
    sel = np.random.default_rng(2).choice(n, 4000, replace=False)
    ora = oracle.Oracle(cfg, pb)
    th = np.asarray(pb.theta0, np.float64)
    oref, nets, st = ora.query(th, pts_np[sel], want_res=True)
    assert st == 0
    do = d.d_out
    for c in range(do):
        assert rel_l2(got[sel, c], oref[:, c]) <= 1e-5, c
    scale = residual_term_scale(query_jets(ora, th, pts_np[sel], nets), cfg)
    assert residual_error(got[sel, do:], oref[:, do:], scale) <= 1e-5


def test_static_query_refuses_more_than_4096_nets():
    Dpinn = _gpu()
    import torch
    from paper_2602_15883_b300 import binding
    lib = binding.load_library()
    cfg = synth.config("beltrami32", unsteady=0, width=32, depth=2, splits=[17, 17, 17, 1],
                       anchor=[0.01, 0.01, 0.01])
    d = Dpinn(cfg)
    assert d.n_nets == 4913
    dummy = torch.zeros(64, device="cuda")
    rc = lib.dpinn_query_static(d.h, dummy.data_ptr(), 4, 0, dummy.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert rc == -1
    assert b"4096" in lib.dpinn_last_error(d.h)
