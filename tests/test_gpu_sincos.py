"""The sine and cosine of the sin activation (the paper's cylinder networks)
against float64 NumPy: the kernels reduce by pi/2 in three parts and sum
Taylor series (dpinn_selftest_sincos runs exactly that code).  Bound: a few
ulp relative to the true value for |x| < 6400, checked densely near 0, at the
multiples of pi/2 (where one of the two nearly vanishes), on random
arguments up to 6400, and NaN for NaN and infinite arguments."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 4 * 2.0 ** -24   # 4 ulp of the result, relative


def _run(x32):
    import torch
    from paper_2602_15883_b300.binding import selftest_sincos
    out = selftest_sincos(torch.from_numpy(x32).cuda()).cpu().numpy().astype(np.float64)
    return out[:, 0], out[:, 1]


def _check(x32):
    s, c = _run(x32)
    x = x32.astype(np.float64)
    rs, rc = np.sin(x), np.cos(x)
    es = np.abs(s - rs) / np.maximum(np.abs(rs), 1e-30)
    ec = np.abs(c - rc) / np.maximum(np.abs(rc), 1e-30)
    assert es.max() <= REL, (float(es.max()), float(x[es.argmax()]))
    assert ec.max() <= REL, (float(ec.max()), float(x[ec.argmax()]))
    return float(es.max()), float(ec.max())


def test_sincos_dense_near_zero_and_random_large():
    rng = np.random.default_rng(0)
    x = np.concatenate([np.linspace(-50.0, 50.0, 400001), rng.uniform(-6400.0, 6400.0, 200000),
                        rng.normal(0.0, 3.0, 200000), [0.0, -0.0, 1e-30, -1e-30, 1e-8, 6399.9]])
    _check(x.astype(np.float32))


def test_sincos_at_multiples_of_half_pi():
    # the float nearest k pi/2 and its neighbours: one of sin, cos is tiny
    k = np.arange(-4000, 4001, dtype=np.float64)
    x = (k * np.pi / 2).astype(np.float32)
    near = np.concatenate([x, np.nextafter(x, np.float32(np.inf)), np.nextafter(x, np.float32(-np.inf))])
    _check(near[np.abs(near) < 6400])


def test_sincos_non_finite_and_empty():
    s, c = _run(np.array([np.nan, np.inf, -np.inf], np.float32))
    assert np.all(np.isnan(s)) and np.all(np.isnan(c))
    s, c = _run(np.zeros(0, np.float32))
    assert s.size == 0 and c.size == 0
