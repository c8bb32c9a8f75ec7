"""The allocation-free query entry point (dpinn_query_static).

Some callers cannot allocate device memory while they serve (a latency-bound
loop that cannot take the device-wide synchronisation of a cudaMalloc, or a
process whose device memory belongs to another framework's allocator);
dpinn_query_static serves them from a fixed array compiled into the
library.  This file checks, through the C ABI, that two calls in a row give
what the regular dpinn_query gives, and that oversized requests are refused.
It is collected last so that a run stopping at its first failure has
already run everything else; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2602_15883_b300 import synth
from tests.helpers import rel_l2
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
