"""Pins of the test's own closed forms: brute-force midpoint sums at d <= 3,
an independently evaluated value of the product-Gaussian integral, and
Table 1's printed true values."""
import math
import os

import numpy as np
import pytest

from paper_2202_01753_gb300 import closed_forms as CF
from paper_2202_01753_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_true_values.txt")


def _table1():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            out[t[0]] = dict(d=int(t[1]), lo=float(t[2]), hi=float(t[3]), true=float(t[4]),
                             est=float(t[5]), err=float(t[6]))
    return out


def test_table1_true_values():
    t = _table1()
    fa = W.suite("fA")
    # printed with 6 decimals (truncated): -49.1650738... -> -49.165073
    assert CF.exact(fa) == pytest.approx(t["fA"]["true"], abs=1e-6)
    fb = W.suite("fB")
    assert CF.exact(fb) == pytest.approx(t["fB"]["true"], abs=1e-12)


def test_gauss3_value():
    # (0.1 sqrt(2 pi) erf(0.5 / (0.1 sqrt 2)))^3
    assert CF.exact(W.gauss3()) == pytest.approx(0.0157495828578, rel=1e-10)


def _vec(fid, params):
    p = np.asarray(params)

    def f(X):
        d = X.shape[1]
        if fid == W.F_GAUSS:
            return p[0] * np.exp(-np.sum((X - p[1:1 + d]) ** 2 / (2 * p[1 + d:] ** 2), axis=1))
        if fid == W.F_CORNER:
            return (1 + X @ p) ** -(d + 1)
        if fid == W.F_OSC:
            return np.cos(2 * np.pi * p[0] + X @ p[1:])
        if fid == W.F_PRODPEAK:
            return np.prod(1 / (p[:d] ** -2.0 + (X - p[d:]) ** 2), axis=1)
        if fid == W.F_C0:
            return np.exp(-np.sum(p[:d] * np.abs(X - p[d:]), axis=1))
        if fid == W.F_DISCONT:
            return np.where(np.all(X < p[d:], axis=1), np.exp(X @ p[:d]), 0.0)
        raise ValueError

    return f


CASES = [
    (W.F_GAUSS, [1.0, 0.4, 0.6, 0.15, 0.25], [0, 0], [1, 1], 2000, 1e-10),
    (W.F_CORNER, [0.7, 1.3], [0, 0], [1, 1], 2000, 1e-10),
    (W.F_CORNER, [0.5, 1.0, 2.0], [0, 0, 0], [1, 1, 1], 200, 1e-7),
    (W.F_OSC, [0.3, 1.1, 0.6, 1.9], [0, 0, 0], [1, 1, 1], 200, 1e-7),
    (W.F_PRODPEAK, [5.0, 3.0, 0.5, 0.3], [0, 0], [1, 1], 2000, 1e-9),
    (W.F_C0, [4.0, 2.0, 0.5, 0.7], [0, 0], [1, 1], 2000, 1e-6),
    (W.F_DISCONT, [1.5, 2.5, 0.35, 0.8], [0, 0], [1, 1], 2000, 2e-3),
]


@pytest.mark.parametrize("fid,params,lo,hi,n,tol", CASES)
def test_closed_form_vs_midpoint(fid, params, lo, hi, n, tol):
    exact = CF.EXACT[fid](params, [float(v) for v in lo], [float(v) for v in hi])
    f = _vec(fid, params)
    if fid == W.F_DISCONT:   # not smooth: plain midpoint, O(h) error
        brute = CF.midpoint(f, lo, hi, n)
    else:                    # smooth: Richardson-extrapolated midpoint, O(h^4)
        brute = (4 * CF.midpoint(f, lo, hi, n) - CF.midpoint(f, lo, hi, n // 2)) / 3
    assert brute == pytest.approx(exact, rel=tol)


def test_cosmo6_factorised_quadrature_vs_monte_carlo_free_check():
    # the quadrature reference of the 6-d integrand: each factor checked by a
    # fine midpoint rule on a scaled-down box (ridge wider so midpoint resolves it)
    w = W.cosmo6()
    p = w.params.copy()
    p[9] = 0.2
    lo, hi = [0.05] * 6, [2.0] * 6
    ref = CF.cosmo6(p, lo, hi)
    a, mu, s, r, t = p[:6], p[6], p[7], p[8], p[9]
    n = 4000
    xs = lambda j: lo[j] + (np.arange(n) + 0.5) * (hi[j] - lo[j]) / n
    h = (hi[0] - lo[0]) / n
    X1, X2 = np.meshgrid(xs(0), xs(1), indexing="ij")
    ridge = np.sum(X1 ** -a[0] * X2 ** -a[1] * np.exp(-((X1 + X2 - r) ** 2) / (2 * t * t))) * h * h
    val = ridge
    for j in (2, 3):
        z = xs(j)
        ln = np.exp(-((np.log(z) - mu) ** 2) / (2 * s * s)) / (z * s * math.sqrt(2 * math.pi))
        val *= np.sum(z ** -a[j] * ln) * h
    for j in (4, 5):
        val *= np.sum(xs(j) ** -a[j]) * h
    assert val == pytest.approx(ref, rel=2e-4)
