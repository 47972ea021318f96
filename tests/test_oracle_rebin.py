"""Pins of the oracle's grid refinement (Adjust-Bin-Bounds of Alg. 2, following
Lepage 1978): cases whose new grid is known in closed form, and the
defining equal-share property."""
import math

import numpy as np
import pytest

import oracle


def uniform(nb):
    return oracle.init_grid(1, nb)[0]


def test_constant_histogram_keeps_uniform_grid():
    for nb in (2, 3, 17, 500, 1024):
        B = uniform(nb)
        st, nB = oracle.rebin_axis(np.full(nb, 3.7), B)
        assert st == oracle.OK
        # edges come from a running sum of nb equal weights: error ~ nb ulp
        assert np.max(np.abs(nB - B)) <= 2 * nb * np.finfo(float).eps
        assert nB[-1] == 1.0


def test_scale_invariance():
    # the histogram is normalised before compression: scaling it changes nothing
    rng = np.random.default_rng(0)
    C = rng.gamma(0.5, size=300)
    B = uniform(300)
    _, a = oracle.rebin_axis(C, B)
    _, b = oracle.rebin_axis(C * 1e12, B)
    assert np.allclose(a, b, rtol=0, atol=1e-15)


def test_alpha_zero_spreads_evenly_over_support():
    # alpha = 0 gives every bin with a nonzero smoothed sum the same weight;
    # smoothing widens a support of bins [lo, hi) by one bin on each side, so
    # the new edges divide [(lo-1)/nb, (hi+1)/nb] into nb equal parts
    nb, lo, hi = 500, 100, 200
    C = np.zeros(nb)
    C[lo:hi] = np.linspace(1, 5, hi - lo)
    _, nB = oracle.rebin_axis(C, uniform(nb), alpha=0.0)
    a, b = (lo - 1) / nb, (hi + 1) / nb
    expect = a + (b - a) * np.arange(1, nb) / nb
    assert np.allclose(nB[:-1], expect, rtol=0, atol=1e-13)
    assert nB[-1] == 1.0


def test_single_interior_bin_spreads_over_three_bins():
    # a histogram in one interior bin smooths into three equal thirds (weights
    # 1/3 each), so the new grid divides those three bins evenly
    nb, k0 = 100, 40
    C = np.zeros(nb)
    C[k0] = 2.0
    _, nB = oracle.rebin_axis(C, uniform(nb), alpha=1.5)
    a, b = (k0 - 1) / nb, (k0 + 2) / nb
    expect = a + (b - a) * np.arange(1, nb) / nb
    assert np.allclose(nB[:-1], expect, rtol=0, atol=1e-13)


def test_first_bin_end_smoothing_and_compression():
    # a histogram in bin 0 smooths to C'_0 = 1/2, C'_1 = 1/3 (end bins average
    # two values, interior bins three); normalised r = (0.6, 0.4); compressed
    # weights ((r - 1)/ln r)^alpha; the new edges split [0, 2/nb] in that ratio
    nb, alpha = 50, 1.5
    C = np.zeros(nb)
    C[0] = 1.0
    _, nB = oracle.rebin_axis(C, uniform(nb), alpha=alpha)
    w0 = ((0.6 - 1) / math.log(0.6)) ** alpha
    w1 = ((0.4 - 1) / math.log(0.4)) ** alpha
    tot = w0 + w1
    expect = []
    for i in range(1, nb):
        t = i * tot / nb
        expect.append((t / w0) / nb if t <= w0 else 1 / nb + ((t - w0) / w1) / nb)
    assert np.allclose(nB[:-1], expect, rtol=0, atol=1e-14)


def test_equal_share_property_random():
    # defining property: with the old bins' weights spread evenly, every new
    # bin holds 1/nb of the total weight.  The weights are recovered from the
    # same rule the closed-form cases above pin down.
    rng = np.random.default_rng(4)
    nb, alpha = 200, 1.5
    B = np.concatenate([np.sort(rng.uniform(0, 1, nb - 1)), [1.0]])
    C = rng.gamma(0.3, size=nb) * (rng.uniform(size=nb) > 0.2)
    st, nB = oracle.rebin_axis(C, B, alpha=alpha)
    assert st == oracle.OK
    sm = np.empty(nb)
    sm[0] = (C[0] + C[1]) / 2
    sm[-1] = (C[-2] + C[-1]) / 2
    sm[1:-1] = (C[:-2] + C[1:-1] + C[2:]) / 3
    r = sm / sm.sum()
    with np.errstate(divide="ignore", invalid="ignore"):
        w = np.where(r > 0, ((r - 1) / np.log(r)) ** alpha, 0.0)
    left = np.concatenate([[0.0], B[:-1]])
    dens = w / (B - left)
    new_left = np.concatenate([[0.0], nB[:-1]])
    for i in range(nb):
        a, b = new_left[i], nB[i]
        ov = np.clip(np.minimum(B, b) - np.maximum(left, a), 0, None)
        assert np.sum(ov * dens) == pytest.approx(w.sum() / nb, rel=1e-9)
    assert np.all(np.diff(np.concatenate([[0.0], nB])) > 0)


def test_heavier_bin_shrinks():
    # importance: raising one bin's sum makes that region's bins narrower
    nb = 100
    C = np.ones(nb)
    C[60] = 50.0
    _, nB = oracle.rebin_axis(C, uniform(nb))
    widths = np.diff(np.concatenate([[0.0], nB]))
    assert widths[59:62].min() < 0.5 / nb
    assert widths[:40].min() > 1.0 / nb


def test_degenerate_histograms():
    B = uniform(10)
    st, nB = oracle.rebin_axis(np.zeros(10), B)
    assert st == 1 and np.array_equal(nB, B)   # no information: unchanged
    C = np.ones(10)
    C[3] = np.inf
    st, nB = oracle.rebin_axis(C, B)
    assert st == oracle.ENONFINITE and np.array_equal(nB, B)
