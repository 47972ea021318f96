"""Exact values of the synthetic workloads' integrals, written from the
mathematics (the true values of the paper's test suite, eqs. 1-6 of Sec. 5,
and of the other families), for accuracy measurements and tests.

These are independent of both the oracle and the CUDA path: every family's
integral over a box is a product of one-dimensional integrals or follows by
inclusion-exclusion, and the closed forms themselves are pinned by
brute-force midpoint sums in tests/test_closed_forms.py.
"""
from __future__ import annotations

import cmath
import itertools
import math

import mpmath
import numpy as np
from scipy import integrate

from . import workloads as W


def gauss(params, lo, hi):
    d = len(lo)
    A, mu, sig = params[0], params[1:1 + d], params[1 + d:1 + 2 * d]
    v = A
    for j in range(d):
        s = sig[j] * math.sqrt(2.0)
        v *= sig[j] * math.sqrt(math.pi / 2.0) * (math.erf((hi[j] - mu[j]) / s) - math.erf((lo[j] - mu[j]) / s))
    return v


def corner(params, lo, hi):
    """(1 + a.x)^-(d+1) over [0,1]^d: (1/(d! prod a)) sum_S (-1)^|S| / (1 + sum_S a)."""
    d = len(lo)
    assert all(l == 0.0 for l in lo) and all(h == 1.0 for h in hi)
    mpmath.mp.dps = 50
    a = [mpmath.mpf(float(v)) for v in params]
    tot = mpmath.mpf(0)
    for r in range(d + 1):
        for S in itertools.combinations(range(d), r):
            tot += (-1) ** r / (1 + sum((a[i] for i in S), mpmath.mpf(0)))
    return float(tot / (mpmath.factorial(d) * mpmath.fprod(a)))


def osc(params, lo, hi):
    """cos(2 pi u + a.x) = Re exp(i(2 pi u + a.x)), a product of 1-d integrals."""
    u, a = params[0], params[1:]
    z = cmath.exp(1j * 2.0 * math.pi * u)
    for j in range(len(lo)):
        z *= (cmath.exp(1j * a[j] * hi[j]) - cmath.exp(1j * a[j] * lo[j])) / (1j * a[j])
    return z.real


def prodpeak(params, lo, hi):
    d = len(lo)
    v = 1.0
    for j in range(d):
        c, w = params[j], params[d + j]
        v *= c * (math.atan(c * (hi[j] - w)) - math.atan(c * (lo[j] - w)))
    return v


def c0(params, lo, hi):
    d = len(lo)
    v = 1.0
    for j in range(d):
        c, w = params[j], params[d + j]
        assert lo[j] <= w <= hi[j]
        v *= (2.0 - math.exp(-c * (w - lo[j])) - math.exp(-c * (hi[j] - w))) / c
    return v


def discont(params, lo, hi):
    d = len(lo)
    v = 1.0
    for j in range(d):
        c, w = params[j], params[d + j]
        top = min(w, hi[j])
        if top <= lo[j]:
            return 0.0
        v *= (math.exp(c * top) - math.exp(c * lo[j])) / c
    return v


def const(params, lo, hi):
    return params[0] * float(np.prod(np.asarray(hi) - np.asarray(lo)))


def cosmo6(params, lo, hi):
    """No closed form: the integrand factorises into a 2-d ridge factor
    (x1, x2), two 1-d lognormal factors (x3, x4) and two power laws (x5, x6),
    each integrated by adaptive quadrature."""
    a, mu, s, r, t = params[:6], params[6], params[7], params[8], params[9]

    def ridge_inner(x1):
        f = lambda x2: x2 ** -a[1] * math.exp(-((x1 + x2 - r) ** 2) / (2 * t * t))
        pts = [r - x1] if lo[1] < r - x1 < hi[1] else None
        return integrate.quad(f, lo[1], hi[1], points=pts, limit=400, epsabs=0, epsrel=1e-13)[0]

    ridge = integrate.quad(lambda x1: x1 ** -a[0] * ridge_inner(x1), lo[0], hi[0], limit=400, epsabs=0,
                           epsrel=1e-12)[0]
    v = ridge
    for j in (2, 3):
        ln = lambda z: math.exp(-((math.log(z) - mu) ** 2) / (2 * s * s)) / (z * s * math.sqrt(2 * math.pi))
        v *= integrate.quad(lambda z: z ** -a[j] * ln(z), lo[j], hi[j], points=[math.exp(mu)], limit=400,
                            epsabs=0, epsrel=1e-13)[0]
    for j in (4, 5):
        v *= (hi[j] ** (1 - a[j]) - lo[j] ** (1 - a[j])) / (1 - a[j])
    return v


def table_weights(n, tlo, thi, a, b):
    """w_i = integral over [a, b] of the i-th piecewise-linear basis function
    ("hat") of n uniform knots on [tlo, thi], extended by constants outside
    the knot range, so that the integral of the linear interpolant of knot
    values v over [a, b] is sum_i w_i v_i."""
    h = (thi - tlo) / (n - 1)
    k = tlo + h * np.arange(n - 1)                  # left knot of every cell
    ta = np.clip((a - k) / h, 0.0, 1.0)
    tb = np.clip((b - k) / h, 0.0, 1.0)
    left = h * ((tb - tb ** 2 / 2) - (ta - ta ** 2 / 2))   # integral of 1 - t over the clipped cell
    right = h * (tb ** 2 / 2 - ta ** 2 / 2)                # integral of t
    w = np.zeros(n)
    w[:-1] += left
    w[1:] += right
    w[0] += max(0.0, min(b, tlo) - a)                # constant extension below the range
    w[-1] += max(0.0, b - max(a, thi))               # and above it
    return w


def table(params, lo, hi, tables):
    """c prod_q T_q over a box, each axis used by at most one factor: the
    product of the factors' integrals (exact for the linear and bilinear
    interpolants, by their basis-function weights) and of the free axes'
    lengths."""
    d = len(lo)
    c, nf = params[0], int(params[1])
    used = set()
    v = c
    for q in range(nf):
        t, a, b = int(params[2 + 3 * q]), int(params[3 + 3 * q]), int(params[4 + 3 * q])
        tb = tables[t]
        vals = np.asarray(tb["values"], dtype=np.float64)
        axes = [a] if b < 0 else [a, b]
        assert not used.intersection(axes), "closed form needs disjoint factor axes"
        used.update(axes)
        tlo, thi = np.atleast_1d(tb["lo"]), np.atleast_1d(tb["hi"])
        w0 = table_weights(vals.shape[0], tlo[0], thi[0], lo[a], hi[a])
        if b < 0:
            v *= float(w0 @ vals)
        else:
            w1 = table_weights(vals.shape[1], tlo[1], thi[1], lo[b], hi[b])
            v *= float(w0 @ (vals @ w1))
    for j in range(d):
        if j not in used:
            v *= hi[j] - lo[j]
    return v


EXACT = {W.F_GAUSS: gauss, W.F_CORNER: corner, W.F_OSC: osc, W.F_PRODPEAK: prodpeak, W.F_C0: c0,
         W.F_DISCONT: discont, W.F_CONST: const, W.F_COSMO6: cosmo6}


def exact(w: W.Workload) -> float:
    if w.fid == W.F_TABLE:
        return table(list(w.params), list(w.lo), list(w.hi), w.meta["tables"])
    return EXACT[w.fid](list(w.params), list(w.lo), list(w.hi))


def midpoint(f, lo, hi, n):
    """Brute-force tensor midpoint rule with n points per axis (vectorised f)."""
    d = len(lo)
    axes = [lo[j] + (np.arange(n) + 0.5) * (hi[j] - lo[j]) / n for j in range(d)]
    grids = np.meshgrid(*axes, indexing="ij")
    X = np.stack([g.reshape(-1) for g in grids], axis=1)
    vol = float(np.prod(np.asarray(hi) - np.asarray(lo)))
    return float(np.mean(f(X))) * vol
