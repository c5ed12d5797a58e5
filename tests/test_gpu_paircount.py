"""Exact GPU pair counts (emulator targets) against the oracle's integer
counts on the same fixed-point coordinates: bit-exact, several uneven sets in
one launch, edge cases (empty, one point, duplicates)."""
import numpy as np
import pytest

import oracle
from paper_1811_05903_gb300 import steps

pytestmark = pytest.mark.gpu


def quantise(x, c, step):
    """Round half away from zero of (x - c) * (1/step), as the library defines it."""
    v = (x - c) * (1.0 / step)
    return np.where(v >= 0, np.floor(v + 0.5), np.ceil(v - 0.5)).astype(np.int32)


def log_edges2(rmin, rmax, nbins, step):
    e = rmin * (rmax / rmin) ** (np.arange(nbins + 1) / nbins)
    return np.ceil((e / step) ** 2).astype(np.int64)


def test_paircount_bit_exact_many_sets():
    steps.load(build_if_missing=True)
    rng = np.random.default_rng(31)
    R, step = 50.0, 50.0 / 2 ** 20
    sizes = [3000, 1, 0, 777, 2048, 4099]
    sets, cen = [], []
    for k, n in enumerate(sizes):
        c = rng.normal(size=3) * 100
        u = rng.uniform(-1, 1, (4 * n + 8, 3))
        pts = u[(u ** 2).sum(1) <= 1][:n] * R + c
        if n > 10:
            pts[5] = pts[4]  # a duplicate pair (d = 0, below the first edge)
        sets.append(pts)
        cen.append(c)
    off = np.concatenate([[0], np.cumsum([len(p) for p in sets])])
    pos = np.concatenate(sets) if len(sets) else np.zeros((0, 3))
    edge2 = log_edges2(0.5, 20.0, 24, step)
    dd = steps.steps_paircount(off, pos, np.array(cen), step, edge2)
    for k, pts in enumerate(sets):
        ref = oracle.paircount(quantise(pts, cen[k], step), edge2) if len(pts) else np.zeros(24, np.uint64)
        np.testing.assert_array_equal(dd[k], ref)
    assert dd[1].sum() == 0 and dd[2].sum() == 0


def test_paircount_poisson_ball_matches_rr():
    """A uniform ball: DD within U-statistic noise of the analytic RR per bin
    (a Poisson term sqrt(RR) plus a term of order RR/sqrt(n))."""
    steps.load(build_if_missing=True)
    rng = np.random.default_rng(32)
    R, n, step = 50.0, 16384, 50.0 / 2 ** 20
    u = rng.uniform(-1, 1, (4 * n, 3))
    pts = u[(u ** 2).sum(1) <= 1][:n] * R
    edges = 0.5 * 40.0 ** (np.arange(25) / 24)
    edge2 = np.ceil((edges / step) ** 2).astype(np.int64)
    dd = steps.steps_paircount(np.array([0, n]), pts, np.zeros((1, 3)), step, edge2)[0].astype(float)
    rr = oracle.rr_ball(n, R, edges)
    big = rr > 100
    assert np.all(np.abs(dd[big] - rr[big]) < 6 * np.sqrt(rr[big]) + 4 * rr[big] / np.sqrt(n))


def test_paircount_rejects_bad_arguments():
    steps.load(build_if_missing=True)
    with pytest.raises(steps.StepsError):
        steps.steps_paircount(np.array([0, 2]), np.zeros((2, 3)), np.zeros((1, 3)), 0.0, np.array([1, 4]))
    with pytest.raises(steps.StepsError):  # 2^29 or more steps from the centre
        steps.steps_paircount(np.array([0, 2]), np.array([[0, 0, 0], [1e12, 0, 0.]]), np.zeros((1, 3)),
                              1e-3, np.array([1, 4]))
