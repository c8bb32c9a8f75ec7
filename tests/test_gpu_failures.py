"""Failure detection on the GPU without faulting it: a bounded device wait
that runs out reports DPINN_ERR_TIMEOUT and leaves the context usable; a
non-finite input surfaces as DPINN_ERR_NONFINITE at the loss read and the
handle recovers once the data are clean."""
import numpy as np
import pytest

from tests.test_gpu_parity import _gpu, small_case

pytestmark = pytest.mark.gpu

TIMEOUT, NONFINITE = -5, -4


def test_bounded_wait_times_out_and_the_context_stays_usable():
    Dpinn = _gpu()
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    assert d.lib.dpinn_selftest_wait(d.h) == TIMEOUT
    assert b"gave up" in d.lib.dpinn_last_error(d.h)
    d.step(2)                       # the handle and the context still work
    loss = d.loss()
    assert np.all(np.isfinite(loss)) and d.get_state()[3] == 2


def test_nan_observation_is_reported_and_the_handle_recovers():
    from paper_2602_15883_b300.binding import POINTS_OBS, DpinnError
    Dpinn = _gpu()
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    bad = np.array(pb.obs_vals, np.float32)
    bad[3, 0] = np.nan
    d.set_points(POINTS_OBS, np.asarray(pb.obs_pts, np.float32), pb.obs_counts, bad)
    d.eval_loss()
    with pytest.raises(DpinnError) as ex:
        d.loss()
    assert ex.value.code == NONFINITE
    d.set_points(POINTS_OBS, np.asarray(pb.obs_pts, np.float32), pb.obs_counts,
                 np.asarray(pb.obs_vals, np.float32))
    d.eval_loss()
    assert np.all(np.isfinite(d.loss()))
