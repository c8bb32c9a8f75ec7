"""The autotuner's axes keep parity: every point tile the library offers
(the FP32 kernels' default and alternate register tiles, the tensor-core
kernels' one), both arithmetics at width 128, and the tuned result, give
losses and gradients that match the FP64 oracle at the same bars as the
default (losses 1e-5, gradients 1e-4, relative L2)."""
import numpy as np
import pytest

import oracle
from tests.helpers import rel_l2
from tests.test_gpu_parity import GRAD_TOL, LOSS_TOL, _gpu, compare_losses, small_case

pytestmark = pytest.mark.gpu

SHAPES = ["kovasznay", "tgv", "unsteady3d_w32", "unsteady3d_w64", "steady3d_w64", "beltrami32", "beltrami128",
          "unsteady2d_w128_deep", "tgv_sin", "cyl2d_w150", "cyl3d_w200"]


def _oracle(cfg, pb):
    return oracle.Oracle(cfg, pb).grad(np.asarray(pb.theta0, np.float64))


def _check(d, ref):
    og, oloss = ref
    d.eval_grad()
    loss, g = d.loss(), d.grad()
    compare_losses(loss, oloss, LOSS_TOL)
    for k in range(d.n_nets):
        assert rel_l2(g[k], og[k]) <= GRAD_TOL, (k, rel_l2(g[k], og[k]))


@pytest.mark.parametrize("name", SHAPES)
def test_every_tile_option_matches_oracle(name):
    Dpinn = _gpu()
    cfg, pb = small_case(name)
    d = Dpinn(cfg)
    d.set_problem(pb)
    precisions = (0, 1) if cfg["width"] == 128 else (0,)
    ref = _oracle(cfg, pb)
    seen = 0
    for p in precisions:
        d.set_precision(p)
        assert d.get_precision() == p
        jo, vo = d.tile_options()
        assert 1 <= len(jo) <= 2 and 1 <= len(vo) <= 2
        for j in range(len(jo)):
            for v in range(len(vo)):
                d.set_tiles(j, v)
                assert d.get_tiles() == ((j, v) if p == 0 else (0, 0))
                assert tuple(d.get_schedule()["tile_points"]) == (jo[j], vo[v])
                _check(d, ref)
                seen += 1
    assert seen >= 1


def test_tile_and_precision_errors():
    Dpinn = _gpu()
    cfg, pb = small_case("tgv")
    d = Dpinn(cfg)
    d.set_problem(pb)
    from paper_2602_15883_b300.binding import DpinnError
    with pytest.raises(DpinnError):
        d.set_tiles(2, 0)          # not an offered tile
    with pytest.raises(DpinnError):
        d.set_precision(1)         # tensor-core kernels need width 128
    assert d.get_precision() == 0
    d.set_tiles(0, 0)
    _check(d, _oracle(cfg, pb))


def test_autotuner_picks_variant_and_tiles_and_keeps_parity(tmp_path, monkeypatch):
    monkeypatch.setenv("DPINN_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    Dpinn = _gpu()
    from paper_2602_15883_b300 import autotune
    cfg, pb = small_case("beltrami32")
    d = Dpinn(cfg)
    d.set_problem(pb)
    n_val = int(pb.obs_counts.sum() + 2 * pb.face_counts.sum())
    res = autotune.autotune(d, pb.n_res, n_val, reps=2, jet_candidates=(1, 4), val_candidates=(1,),
                            precisions=(0, 1))
    assert not res["cached"] and res["trials"] >= 5
    assert set(res["precision_ms"]) == {"0", "1"}
    assert d.get_precision() == res["precision"]
    assert tuple(d.get_schedule()["tile_points"]) == tuple(res["tile_points"])
    assert d.get_tiles() == ((res["jet_tile"], res["val_tile"]) if res["precision"] == 0 else (0, 0))
    _check(d, _oracle(cfg, pb))
    # a fresh handle takes the cached choice
    d2 = Dpinn(cfg)
    d2.set_problem(pb)
    again = autotune.autotune(d2, pb.n_res, n_val, precisions=(0, 1))
    assert again["cached"] and d2.get_precision() == res["precision"]
    assert tuple(d2.get_schedule()["tile_points"]) == tuple(res["tile_points"])
