"""Pins of the oracle's geometry and map (Alg. 1 map step, Alg. 2 geometry):
exact rationals, the defining property of g, and the identities a uniform
grid must satisfy."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2202_01753_gb300 import workloads as W


@pytest.mark.parametrize("d,ncall", [(1, 10), (2, 100), (3, 2 ** 20), (6, 10 ** 8), (8, 10 ** 9),
                                     (10, 10 ** 9), (12, 10 ** 7), (5, 3)])
def test_geometry_defining_property(d, ncall):
    g, m, p = oracle.geometry(d, ncall)
    assert m == g ** d
    half = ncall // 2
    assert g == 1 or g ** d <= half
    assert (g + 1) ** d > min(half, 2 ** 32 - 1) or (g + 1) * 500 > 2 ** 31
    assert p == max(ncall // m, 2)


def test_geometry_matches_printed_configs():
    assert oracle.geometry(3, 2 ** 20, 4) == (4, 64, 16384)
    assert oracle.geometry(6, 10 ** 8) == (19, 47045881, 2)
    assert oracle.geometry(8, 10 ** 9) == (12, 429981696, 2)
    assert oracle.geometry(10, 10 ** 9) == (7, 282475249, 3)


def test_geometry_rejects():
    for args in [(0, 100), (13, 100), (3, 1)]:
        with pytest.raises(ValueError):
            oracle.geometry(*args)
    with pytest.raises(ValueError):
        oracle.geometry(2, 100, g_override=2 ** 20)  # m would exceed 32 bits


def test_bin_of_is_exact_rational():
    rng = np.random.default_rng(5)
    for _ in range(3000):
        g = int(rng.integers(1, 5000))
        nb = int(rng.integers(2, 1025))
        c = int(rng.integers(0, g))
        w = int(rng.integers(0, 2 ** 32))
        t = Fraction(nb) * (c + Fraction(2 * w + 1, 2 ** 33)) / g
        k, phi = oracle.bin_of(c, w, g, nb)
        assert k == int(t)  # floor (t > 0)
        assert 0 <= k < nb
        assert abs(phi - float(t - k)) <= 2.0 ** -52
        assert 0.0 <= phi < 1.0


def test_bin_of_extremes():
    # the corners of the word range never leave the cube or the grid
    for g in (1, 2, 7, 19, 4096):
        for nb in (2, 3, 500, 1024):
            k, phi = oracle.bin_of(g - 1, 2 ** 32 - 1, g, nb)
            assert k == nb - 1 and phi < 1.0
            k, phi = oracle.bin_of(0, 0, g, nb)
            assert k == 0 and phi > 0.0


def _uniform_map_problem(d, g_override, fid=W.F_CONST, params=(1.0,)):
    lo = np.linspace(-1.0, 0.5, d)
    hi = lo + np.linspace(0.5, 3.0, d)
    return oracle.Problem(fid, params, lo, hi, ncall=2 * g_override ** d * 4, g_override=g_override), lo, hi


def test_uniform_grid_constant_is_exact():
    # f = 1 on the uniform grid: every F equals the volume (up to the rounding
    # of the edges (k+1)/nb), so the estimate is the volume and the variance is
    # zero to rounding
    for d in (1, 3, 6):
        pb, lo, hi = _uniform_map_problem(d, 3)
        B = oracle.init_grid(d, pb.nb)
        sums, C, H, st = pb.vsample(B, it=0, adjust=True, hits=True)
        vol = float(np.prod(hi - lo))
        assert st == oracle.OK
        assert sums[0] / pb.m == pytest.approx(vol, rel=1e-14)
        assert np.sqrt(sums[1]) / pb.m <= 1e-15 * vol
        # every sample lands in exactly one bin per axis; F^2 = vol^2 each
        N = pb.m * pb.p
        assert np.all(H.sum(axis=1) == N)
        assert np.allclose(C.sum(axis=1), N * vol * vol, rtol=1e-13)


def test_uniform_grid_is_plain_stratified_monte_carlo():
    # On the uniform grid the map is x = lo + (hi - lo) y and J = volume, so a
    # pass reduces to plain stratified Monte Carlo: per cube, the sample mean
    # and (numpy's) unbiased variance of f(x) * volume over its p points.
    d, g = 2, 3
    a = np.array([0.7, 1.9])
    lo, hi = np.array([0.0, -1.0]), np.array([2.0, 0.5])
    vol = float(np.prod(hi - lo))
    pb = oracle.Problem(W.F_CORNER, a, lo, hi, ncall=g ** d * 37, g_override=g, seed=99)
    B = oracle.init_grid(d, pb.nb)
    sums, _, _, _ = pb.vsample(B, it=4, adjust=False)
    means, vars_ = [], []
    for c in range(pb.m):
        digits = [c % g, c // g]
        F = []
        for s in range(pb.p):
            w = oracle.sample_words(99, 4, c, s, d).astype(np.float64)
            y = (np.array(digits) + (w + 0.5) / 2.0 ** 32) / g
            x = lo + (hi - lo) * y
            F.append(vol * (1.0 + a @ x) ** -(d + 1))
        F = np.array(F)
        means.append(F.mean())
        vars_.append(F.var(ddof=1) / pb.p)
    assert sums[0] == pytest.approx(np.sum(means), rel=1e-13)
    assert sums[1] == pytest.approx(np.sum(vars_), rel=1e-11)
    assert sums[2] == pytest.approx(np.sum(np.abs(means)), rel=1e-13)


def test_map_continuous_at_edges_and_monotone():
    # a random non-uniform grid: x(y) increases with y and is continuous across
    # bin edges (evaluated just left and right of every edge)
    rng = np.random.default_rng(1)
    nb = 50
    edges = np.sort(rng.uniform(0, 1, nb - 1))
    B = np.concatenate([edges, [1.0]])
    lo, hi = 2.0, 5.0

    def x_of(k, phi):
        left = B[k - 1] if k else 0.0
        return lo + (hi - lo) * (left + (B[k] - left) * phi)

    for k in range(nb - 1):
        assert x_of(k, 1.0) == pytest.approx(x_of(k + 1, 0.0), abs=1e-15)
    xs = [x_of(k, phi) for k in range(nb) for phi in np.linspace(0, 1, 7)]
    assert np.all(np.diff(xs) >= -1e-15)


def test_jacobian_integrates_to_volume():
    # with any fixed grid, the mean over a full stratified pass of J estimates
    # the volume (f = 1) within its error; bins finer than the sub-cubes so
    # that J varies inside a cube
    rng = np.random.default_rng(2)
    d, nb = 2, 200
    B = np.stack([np.concatenate([np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(d)])
    pb = oracle.Problem(W.F_CONST, [1.0], [0.0, 1.0], [2.0, 4.0], ncall=2000, nb=nb)
    assert pb.g < nb
    sums, _, _, _ = pb.vsample(B, it=0, adjust=False)
    est = sums[0] / pb.m
    sig = np.sqrt(sums[1]) / pb.m
    assert sig > 0
    assert abs(est - 6.0) < 5 * sig


def test_cube_coarser_than_bins_is_exact_for_constants():
    # when every sub-cube lies inside one bin per axis (g a multiple of nb),
    # J is constant on each cube and f = 1 is integrated exactly
    rng = np.random.default_rng(3)
    d, nb = 2, 20
    B = np.stack([np.concatenate([np.sort(rng.uniform(0, 1, nb - 1)), [1.0]]) for _ in range(d)])
    pb = oracle.Problem(W.F_CONST, [1.0], [0.0, 1.0], [2.0, 4.0], ncall=20000, nb=nb)
    assert pb.g % nb == 0
    sums, _, _, _ = pb.vsample(B, it=0, adjust=False)
    assert sums[0] / pb.m == pytest.approx(6.0, rel=1e-13)
    assert sums[1] == 0.0
