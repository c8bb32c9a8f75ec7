"""Host logic of the serving loop: FIFO admission under slot and memory caps."""
import numpy as np

from paper_2602_15883_b300.serve import Request, plan_batch, request_bytes


def _req(n, res=False):
    return Request(pts=np.zeros((n, 4), np.float32), want_residual=res)


def test_fifo_prefix_within_caps():
    w = lambda r: 8 if r.want_residual else 4
    pend = [_req(100), _req(200, True), _req(50), _req(1000)]
    take, mem = plan_batch(pend, max_points=400, budget_left=10 ** 9, d_in=4, width_of=w)
    assert [r.n for r in take] == [100, 200, 50]
    assert mem == request_bytes(100, 4, 4) + request_bytes(200, 4, 8) + request_bytes(50, 4, 4)


def test_memory_budget_blocks_admission_in_order():
    w = lambda r: 4
    pend = [_req(100), _req(10), _req(10)]
    budget = request_bytes(100, 4, 4) + request_bytes(10, 4, 4) - 1
    take, mem = plan_batch(pend, max_points=10 ** 6, budget_left=budget, d_in=4, width_of=w)
    assert [r.n for r in take] == [100]     # the next one does not fit; no overtaking
    take, mem = plan_batch(pend, max_points=10 ** 6, budget_left=0, d_in=4, width_of=w)
    assert take == [] and mem == 0


def test_request_bytes_counts_points_outputs_and_routing():
    assert request_bytes(1000, 4, 8) == 1000 * 4 * (4 + 8 + 2)
