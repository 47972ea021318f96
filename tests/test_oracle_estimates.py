"""Pins of the oracle's whole driver (Alg. 2) against closed forms,
invariants and statistics (Sec. 5.1's accuracy protocol, scaled down)."""
import numpy as np
import pytest

from paper_2202_01753_gb300 import closed_forms as CF
import oracle
from paper_2202_01753_gb300 import workloads as W


def run(w, **kw):
    args = dict(ita=w.ita, nb=w.nb, g_override=w.g_override, seed=w.seed, rel_tol=w.rel_tol, abs_tol=w.abs_tol)
    args.update(kw)
    return oracle.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, **args)


def test_gauss3_full_config():
    w = W.gauss3()
    r = run(w)
    assert r["status"] == oracle.ENOCONV and r["iterations"] == 10   # rel_tol 0: runs all iterations
    assert (r["g"], r["m"], r["p"]) == (4, 64, 16384)
    exact = CF.exact(w)
    assert abs(r["estimate"] - exact) < 4 * r["sigma"]
    # adaptation: the per-iteration error falls by an order of magnitude
    s = np.sqrt(r["trace_var"])
    assert s[-1] < s[0] / 10
    assert r["chi2_dof"] < 3.0
    B = r["grid"]
    assert np.all(np.diff(B, axis=1) > 0) and np.all(B[:, -1] == 1.0)
    # the grid concentrates where the Gaussian peaks (centre bins narrower)
    widths = np.diff(np.concatenate([np.zeros((3, 1)), B], axis=1), axis=1)
    assert np.all(widths[:, 240:260].mean(axis=1) < widths[:, :20].mean(axis=1))


SUITE = [
    ("f1", 3, 200_000), ("f2", 3, 200_000), ("f3", 4, 200_000), ("f4", 3, 200_000),
    ("f5", 3, 200_000), ("f6", 3, 200_000), ("fA", None, 400_000), ("fB", None, 400_000),
]


@pytest.mark.parametrize("name,d,ncall", SUITE)
def test_paper_suite_against_closed_forms(name, d, ncall):
    w = W.suite(name, d, ncall=ncall, itmax=8, seed=3)
    r = run(w)
    assert r["status"] in (oracle.OK, oracle.ENOCONV)
    exact = CF.exact(w)
    assert abs(r["estimate"] - exact) < 5 * r["sigma"] + 1e-12 * abs(exact)


@pytest.mark.parametrize("make", [W.corner8, W.osc10])
def test_mixed_configs_scaled_down_against_closed_forms(make):
    w = make().scaled(300_000, itmax=6)
    r = run(w)
    exact = CF.exact(w)
    assert abs(r["estimate"] - exact) < 5 * r["sigma"]


def test_cosmo6_scaled_down_against_quadrature():
    w = W.cosmo6().scaled(300_000, itmax=8)
    r = run(w)
    ref = CF.exact(w)
    assert abs(r["estimate"] - ref) < 5 * r["sigma"]


def test_histogram_invariants():
    # every sample adds F^2 once per axis, so the axis totals agree; every
    # sample lands in exactly one bin per axis
    w = W.suite("f4", 3, ncall=50_000)
    pb = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, seed=5)
    B = oracle.init_grid(3, pb.nb)
    sums, C, H, st = pb.vsample(B, it=0, adjust=True, hits=True)
    tot = C.sum(axis=1)
    assert np.allclose(tot, tot[0], rtol=1e-13)
    assert np.all(H.sum(axis=1) == pb.m * pb.p)


def test_sigma_shrinks_with_ncall():
    # fixed uniform grid (no adjusting iterations): the error falls at least
    # like ncall^-1/2
    w = W.suite("f4", 2, itmax=1)
    s = []
    for n in (10_000, 160_000):
        r = run(w.scaled(n), ita=0)
        s.append(r["sigma"])
    assert s[1] < s[0] / 4 * 1.2


def test_reproducible_and_seeded():
    w = W.suite("f3", 3, ncall=20_000, itmax=4)
    a, b, c = run(w, seed=1), run(w, seed=1), run(w, seed=2)
    assert a["estimate"] == b["estimate"] and np.array_equal(a["grid"], b["grid"])
    assert a["estimate"] != c["estimate"]


def test_coverage_over_seeds():
    # Sec. 5.1 protocol in miniature: over many seeds the true value lies
    # within 2 sigma for about 95% of runs
    w = W.suite("f4", 2, ncall=4_000, itmax=6)
    exact = CF.exact(w)
    hits = 0
    n = 120
    for seed in range(n):
        r = run(w, seed=seed)
        hits += abs(r["estimate"] - exact) <= 2 * r["sigma"]
    assert hits / n > 0.85


def test_convergence_stops_early():
    w = W.gauss3()
    r = run(w.scaled(2 ** 16), rel_tol=1e-3)
    assert r["status"] == oracle.OK and r["converged"]
    assert 2 <= r["iterations"] < 10
    assert r["sigma"] <= 1e-3 * abs(r["estimate"])


def test_nonfinite_is_reported():
    # F^2 overflows the histogram: the refinement refuses the grid
    w = W.suite("f4", 2, ncall=2_000, itmax=3)
    p = w.params.copy()
    p[0] = 1e300
    r = oracle.integrate(w.fid, p, w.lo, w.hi, w.ncall, w.itmax)
    assert r["status"] == oracle.ENONFINITE
