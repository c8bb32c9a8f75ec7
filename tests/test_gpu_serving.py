"""Continuous batching: results are the same alone and in a Poisson mix,
admission respects the memory cap, batches overlap, bad requests fail alone."""
import numpy as np
import pytest

import oracle
from paper_2602_15883_b300 import synth
from tests.helpers import rel_l2
from tests.test_gpu_parity import _gpu

pytestmark = pytest.mark.gpu


def _server(slots=3, mem_cap=1 << 30, max_batch=1 << 18):
    Dpinn = _gpu()
    from paper_2602_15883_b300.serve import Server
    cfg = synth.config("beltrami32")
    pb = synth.make_problem(cfg, seed=0, res_counts=[64] * 32, obs_counts=[16] * 32, face_counts=[8] * 72,
                            bias_std=0.1)
    d = Dpinn(cfg)
    d.set_problem(pb)
    return cfg, pb, d, Server(d, slots=slots, mem_cap_bytes=mem_cap, max_batch_points=max_batch).start()


def test_alone_equals_in_the_mix_and_matches_oracle():
    from paper_2602_15883_b300.serve import latency_summary, poisson_load
    cfg, pb, d, srv = _server()
    try:
        probe_v = synth.query_points(cfg, 3000, seed=11)
        probe_r = synth.query_points(cfg, 2000, seed=12)
        a_v = srv.submit(probe_v, False)
        a_r = srv.submit(probe_r, True)
        a_v.done.wait(); a_r.done.wait()
        # the same requests in the middle of a Poisson stream of others
        import threading
        box = {}
        t = threading.Thread(target=lambda: box.setdefault(
            "reqs", poisson_load(srv, cfg, rate_hz=400, duration_s=0.6, seed=3, n_min=500, n_max=60000,
                                 residual_fraction=0.3)))
        t.start()
        import time
        time.sleep(0.25)
        b_v = srv.submit(probe_v, False)
        b_r = srv.submit(probe_r, True)
        t.join()
        b_v.done.wait(); b_r.done.wait()
        mix = box["reqs"]
        assert len(mix) > 100 and all(r.error is None for r in mix)
        np.testing.assert_array_equal(a_v.result, b_v.result)
        np.testing.assert_array_equal(a_r.result, b_r.result)
        summ = latency_summary(mix)
        assert summ["p99_ms"] >= summ["p50_ms"] > 0
        assert srv.max_concurrent >= 2
        # against the regular query and the oracle
        import torch
        ref_v = d.query(torch.from_numpy(probe_v).cuda()).cpu().numpy()
        np.testing.assert_array_equal(a_v.result, ref_v)
        ora = oracle.Oracle(cfg, pb)
        o_v, _, st = ora.query(np.asarray(pb.theta0, np.float64), probe_v)
        assert st == 0 and rel_l2(a_v.result, o_v) <= 1e-5
    finally:
        srv.stop()


def test_memory_cap_is_respected_and_everything_completes():
    """All device memory the server allocates (every slot's buffers and query
    contexts, measured by the device's free memory) stays under the cap, with
    a 1M-point residual request - larger than a slot, so served in chunks -
    in a mix of others; every result equals the regular query's."""
    import threading
    import time
    import torch
    from paper_2602_15883_b300.serve import Server
    Dpinn = _gpu()
    cfg = synth.config("beltrami32")
    pb = synth.make_problem(cfg, seed=0, res_counts=[64] * 32, obs_counts=[16] * 32, face_counts=[8] * 72,
                            bias_std=0.1)
    d = Dpinn(cfg)
    d.set_problem(pb)
    big_pts = synth.query_points(cfg, 1 << 20, seed=40)
    ref_big = d.query(torch.from_numpy(big_pts).cuda(), want_residual=True).cpu().numpy()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0 = torch.cuda.mem_get_info()[0]
    cap = 96 << 20
    srv = Server(d, slots=3, mem_cap_bytes=cap, max_batch_points=None).start()
    assert srv.device_bytes <= cap and srv.max_points < (1 << 20)
    peak = [0]
    stop = threading.Event()

    def watch():
        while not stop.is_set():
            peak[0] = max(peak[0], free0 - torch.cuda.mem_get_info()[0])
            time.sleep(0.0005)
    w = threading.Thread(target=watch)
    w.start()
    try:
        mix = [srv.submit(synth.query_points(cfg, n, seed=n), bool(n % 3 == 0)) for n in
               [30000, 39000, 1000, 25000, 12000, 40000, 5000]]
        big = srv.submit(big_pts, True)
        mix += [srv.submit(synth.query_points(cfg, n, seed=n + 1), bool(n % 2)) for n in (3000, 90001, 7)]
        for r in mix + [big]:
            r.done.wait()
        assert all(r.error is None and r.result.shape[0] == r.n for r in mix)
        assert big.error is None and len(big.chunks) >= 4
        np.testing.assert_array_equal(big.result, ref_big)
        for r in mix[:2]:
            ref = d.query(torch.from_numpy(r.pts).cuda(), want_residual=r.want_residual).cpu().numpy()
            np.testing.assert_array_equal(r.result, ref)
        assert 0 < srv.max_in_flight_bytes <= cap
    finally:
        stop.set()
        w.join()
        srv.stop()
    assert 0 < peak[0] <= cap, (peak[0], cap)


def test_bad_requests_fail_alone():
    cfg, pb, d, srv = _server()
    try:
        bad = synth.query_points(cfg, 100, seed=1)
        bad[5, 0] = 3.0
        r_bad = srv.submit(bad)
        big = srv.submit(np.zeros(((1 << 18) + 1, 4), np.float32))    # two slot-sized chunks
        good = srv.submit(synth.query_points(cfg, 100, seed=2))
        for r in (r_bad, big, good):
            r.done.wait()
        assert r_bad.error and "outside" in r_bad.error
        assert big.error is None and big.result.shape == ((1 << 18) + 1, 4) and len(big.chunks) == 2
        assert good.error is None and good.result.shape == (100, 4)
    finally:
        srv.stop()


def test_cancelled_requests_end_alone():
    cfg, pb, d, srv = _server(slots=1)
    try:
        first = srv.submit(synth.query_points(cfg, 200000, seed=3), True)     # occupies the only slot
        waiting = srv.submit(synth.query_points(cfg, 1000, seed=4))
        other = srv.submit(synth.query_points(cfg, 1000, seed=5))
        assert srv.cancel(waiting)
        for r in (first, waiting, other):
            r.done.wait()
        assert waiting.error == "cancelled" and waiting.result is None
        assert first.error is None and first.result.shape == (200000, 8)
        assert other.error is None and other.result.shape == (1000, 4)
        assert not srv.cancel(other)          # already finished
    finally:
        srv.stop()


def test_caller_buffers_receive_the_same_results():
    cfg, pb, d, srv = _server(slots=2)
    try:
        pts_v = synth.query_points(cfg, 5000, seed=21)
        pts_r = synth.query_points(cfg, 3000, seed=22)
        a = srv.submit(pts_v)
        b = srv.submit(pts_r, True)
        ov = np.full((5000, 4), -7.0, np.float32)
        orr = np.full((3000, 8), -7.0, np.float32)
        c = srv.submit(pts_v, out=ov)
        e = srv.submit(pts_r, True, out=orr)
        for r in (a, b, c, e):
            r.done.wait()
        assert c.result is ov and e.result is orr
        np.testing.assert_array_equal(ov, a.result)
        np.testing.assert_array_equal(orr, b.result)
        with pytest.raises(ValueError):
            srv.submit(pts_v, out=np.zeros((5000, 8), np.float32))   # residual width for a value query
        with pytest.raises(ValueError):
            srv.submit(pts_v, out=np.zeros((5000, 4), np.float64))
    finally:
        srv.stop()


def test_cancelling_a_chunked_request():
    cfg, pb, d, srv = _server(slots=1, max_batch=1 << 16)
    try:
        first = srv.submit(synth.query_points(cfg, 200000, seed=3), True)   # 4 chunks, the slot stays busy
        big = srv.submit(synth.query_points(cfg, 300000, seed=6))           # 5 chunks, waiting
        after = srv.submit(synth.query_points(cfg, 1000, seed=7))
        assert srv.cancel(big)
        for r in (first, big, after):
            r.done.wait()
        assert big.error == "cancelled" and big.result is None
        assert first.error is None and first.result.shape == (200000, 8)
        assert after.error is None and after.result.shape == (1000, 4)
    finally:
        srv.stop()
