"""Pins of the oracle's collocation sampler (per-step resampling).

The generator is SplitMix64 used as counter-based streams; it is pinned to
the generator's published reference outputs, and the sampled points to the
properties the method needs: inside each net's cell, uniform, independent
across axes, steps, nets and seeds, reproducible.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2602_15883_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")


def test_splitmix64_matches_published_reference_outputs():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        n, hx = line.split()
        assert oracle.splitmix64_nth(0, int(n)) == int(hx, 16), n


def _cfg():
    return synth.config("beltrami32", splits=[2, 1, 1, 2])


def test_points_lie_in_their_cells_and_counts_are_respected():
    cfg = _cfg()
    o = oracle.Oracle(cfg)
    counts = np.array([0, 7, 300, 1])
    pts = o.sample(3, 5, counts)
    assert pts.shape == (counts.sum(), o.d_in) and pts.dtype == np.float32
    row = 0
    for k, n in enumerate(counts):
        blk = pts[row:row + n]
        row += n
        lo = o.box_lo[k, :o.d_in].astype(np.float32)
        hi = o.box_hi[k, :o.d_in].astype(np.float32)
        assert np.all(blk >= lo) and np.all(blk <= hi)


@pytest.mark.parametrize("t", [0, 1, 17])
def test_points_are_uniform_and_independent_across_axes(t):
    cfg = _cfg()
    o = oracle.Oracle(cfg)
    n = 20000
    counts = np.array([n, 0, 0, n])
    pts = o.sample(11, t, counts).astype(np.float64)
    for k, blk in ((0, pts[:n]), (3, pts[n:])):
        u = (blk - o.box_lo[k, :o.d_in]) / (o.box_hi[k, :o.d_in] - o.box_lo[k, :o.d_in])
        for d in range(o.d_in):
            assert stats.kstest(u[:, d], "uniform").pvalue > 1e-3, (k, d)
        c = np.corrcoef(u.T)
        off = c[~np.eye(o.d_in, dtype=bool)]
        assert np.all(np.abs(off) < 5 / np.sqrt(n))


def test_streams_are_reproducible_and_distinct():
    cfg = _cfg()
    o = oracle.Oracle(cfg)
    counts = np.array([50, 50, 50, 50])
    a = o.sample(1, 0, counts)
    np.testing.assert_array_equal(a, o.sample(1, 0, counts))
    assert not np.array_equal(a, o.sample(1, 1, counts))        # another step
    assert not np.array_equal(a, o.sample(2, 0, counts))        # another seed
    # the nets draw different streams: normalised coordinates differ
    u = [(a[50 * k:50 * (k + 1)] - o.box_lo[k, :o.d_in]) / (o.box_hi[k, :o.d_in] - o.box_lo[k, :o.d_in])
         for k in range(4)]
    assert np.max(np.abs(u[0] - u[1])) > 0.1
    # a net's first points do not depend on how many points it draws
    b = o.sample(1, 0, np.array([10, 50, 50, 50]))
    np.testing.assert_array_equal(b[:10], a[:10])
