"""Pins of the oracle's TABLE family (integrands that read interpolation
tables, the paper's stateful integrands of Sec. 6.1) and of the closed form
used to check it.  The interpolant of a table sampled from a linear
(bilinear) function is that function, knots reproduce their values, points
outside the range take the edge values, and the estimates of whole runs
agree with the exact integral of the interpolant, whose code is itself
pinned by brute-force midpoint sums."""
import numpy as np
import pytest

import oracle
from paper_2202_01753_gb300 import closed_forms as CF
from paper_2202_01753_gb300 import workloads as W


def _set(tables):
    oracle.set_tables(tables)


def _f(params, x):
    return oracle.integrand(W.F_TABLE, params, x)


def test_linear_table_is_exact_and_clamps():
    n = 65                                          # knots 1/64 apart: exact knot positions
    k = np.linspace(0.0, 2.0, n)
    _set([dict(ndim=1, values=3.0 - 1.25 * k, lo=0.0, hi=2.0)])
    p = [2.0, 1, 0, 0, -1]
    rng = np.random.default_rng(1)
    for x in rng.uniform(0.0, 2.0, 200):
        assert _f(p, [x]) == pytest.approx(2.0 * (3.0 - 1.25 * x), rel=1e-15, abs=1e-15)
    for i in (0, 17, 64):                           # knots give their values exactly
        assert _f(p, [k[i]]) == 2.0 * (3.0 - 1.25 * k[i])
    assert _f(p, [-5.0]) == 2.0 * 3.0 and _f(p, [9.0]) == 2.0 * (3.0 - 2.5)


def test_bilinear_table_is_exact_on_its_axes():
    n0, n1 = 17, 33
    X, Y = np.meshgrid(np.linspace(0, 1, n0), np.linspace(-1, 1, n1), indexing="ij")
    V = 0.5 + X - 2.0 * Y + 3.0 * X * Y
    _set([dict(ndim=2, values=V, lo=(0.0, -1.0), hi=(1.0, 1.0))])
    p = [1.0, 1, 0, 2, 0]                           # T(x_2, x_0) of a 3-d point
    rng = np.random.default_rng(2)
    for _ in range(200):
        x = rng.uniform([-1, 0, 0], [1, 1, 1])
        want = 0.5 + x[2] - 2.0 * x[0] + 3.0 * x[2] * x[0]
        assert _f(p, x) == pytest.approx(want, rel=1e-14, abs=1e-14)


def test_product_of_factors_and_param_validation():
    k = np.linspace(0, 1, 9)
    _set([dict(ndim=1, values=1 + k, lo=0.0, hi=1.0), dict(ndim=1, values=2 - k, lo=0.0, hi=1.0),
          dict(ndim=2, values=np.ones((3, 3)), lo=(0, 0), hi=(1, 1))])
    x = np.array([0.25, 0.5, 0.75])
    assert _f([1.5, 2, 0, 0, -1, 1, 2, -1], x) == pytest.approx(1.5 * 1.25 * 1.25, rel=1e-15)
    assert oracle.table_params_ok([1.5, 2, 0, 0, -1, 1, 2, -1], 3)
    assert not oracle.table_params_ok([1.5, 2, 0, 0, -1, 1, 2], 3)        # wrong length
    assert not oracle.table_params_ok([1.5, 1, 3, 0, -1], 3)              # no table 3
    assert not oracle.table_params_ok([1.5, 1, 0, 0, 1], 3)               # 1-D table given two axes
    assert not oracle.table_params_ok([1.5, 1, 2, 1, -1], 3)              # 2-D table given one axis
    assert not oracle.table_params_ok([1.5, 1, 2, 1, 1], 3)               # the same axis twice
    assert not oracle.table_params_ok([1.5, 1, 0, 3, -1], 3)              # no axis 3
    assert not oracle.table_params_ok([1.5, 1.5, 0, 0, -1], 3)            # fractional count


@pytest.mark.parametrize("a,b", [(0.0, 1.0), (0.13, 0.77), (-0.5, 1.3), (0.5, 0.5 + 1e-3)])
def test_closed_form_weights_against_midpoint(a, b):
    n = 11
    rng = np.random.default_rng(3)
    v = rng.uniform(-1, 2, n)
    w = CF.table_weights(n, 0.0, 1.0, a, b)
    k = np.linspace(0.0, 1.0, n)
    m = 200_000
    x = a + (np.arange(m) + 0.5) * (b - a) / m
    brute = np.interp(np.clip(x, 0.0, 1.0), k, v).mean() * (b - a)
    assert float(w @ v) == pytest.approx(brute, rel=1e-9, abs=1e-12)


def test_closed_form_2d_against_midpoint():
    rng = np.random.default_rng(4)
    V = rng.uniform(0, 1, (5, 7))
    tables = [dict(ndim=2, values=V, lo=(0.0, 0.0), hi=(1.0, 2.0))]
    params = [1.0, 1, 0, 0, 1]
    lo, hi = [0.1, 0.3], [0.9, 1.7]
    got = CF.table(params, lo, hi, tables)
    _set(tables)
    m = 400
    xs = lo[0] + (np.arange(m) + 0.5) * (hi[0] - lo[0]) / m
    ys = lo[1] + (np.arange(m) + 0.5) * (hi[1] - lo[1]) / m
    brute = np.mean([[_f(params, [x, y]) for y in ys[::8]] for x in xs[::8]]) * (hi[0] - lo[0]) * (hi[1] - lo[1])
    assert got == pytest.approx(brute, rel=2e-3)
    # midpoint in full on the bilinear interpolant via numpy (exact per-cell quadratic, error O(1/m^2))
    k0, k1 = np.linspace(0, 1, 5), np.linspace(0, 2, 7)
    A = np.array([np.interp(ys, k1, V[i]) for i in range(5)])          # interpolate along axis 1
    B = np.array([np.interp(xs, k0, A[:, j]) for j in range(m)])       # then along axis 0
    assert got == pytest.approx(B.mean() * (hi[0] - lo[0]) * (hi[1] - lo[1]), rel=1e-5)


@pytest.mark.parametrize("seed", [5, 6])
def test_oracle_estimate_of_table6_small(seed):
    w = W.table6(seed=seed, n2=257, n1=4097, ncall=60_000, itmax=6)
    oracle.set_tables(w.meta["tables"])
    r = oracle.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, seed=w.seed)
    exact = CF.exact(w)
    assert r["status"] in (0, 5)
    assert abs(r["estimate"] - exact) <= 4 * r["sigma"], (r["estimate"], exact, r["sigma"])
    assert r["sigma"] < 0.05 * abs(exact)
