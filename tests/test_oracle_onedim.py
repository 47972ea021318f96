"""Pins of the oracle's m-Cubes1D variant (Sec. 3, "The m-Cubes1D variant":
all axes share one set of bin boundaries, so only axis 0 keeps a histogram
and is rebinned).  Each test reduces the variant to parts of the oracle that
are pinned elsewhere (V-Sample, the rebinning of one axis, the m-Cubes
driver) or to the closed forms of the paper's symmetric integrands."""
import numpy as np
import pytest

from paper_2202_01753_gb300 import closed_forms as CF
import oracle
from paper_2202_01753_gb300 import workloads as W


def _run(w, **kw):
    args = dict(nb=w.nb, g_override=w.g_override, seed=w.seed, rel_tol=w.rel_tol, abs_tol=w.abs_tol)
    args.update(kw)
    return oracle.integrate(w.fid, w.params, w.lo, w.hi, w.ncall, w.itmax, **args)


def test_one_axis_is_plain_mcubes():
    """With d = 1 there is one axis: the variant is m-Cubes itself."""
    w = W.suite("f4", d=1, ncall=4000, itmax=6)
    a, b = _run(w), _run(w, one_dim=True)
    for k in ("estimate", "sigma", "chi2_dof", "iterations"):
        assert a[k] == b[k]
    assert np.array_equal(a["trace_I"], b["trace_I"]) and np.array_equal(a["grid"], b["grid"])
    assert np.array_equal(a["hist"], b["hist"])


@pytest.mark.parametrize("name,d", [("f2", 4), ("f5", 3), ("f3", 3)])
def test_axis0_histogram_is_the_plain_one(name, d):
    """On a grid whose rows are equal, the variant's V-Sample draws the same
    samples and gives the same sums and the same axis-0 histogram (and hit
    counts) as plain V-Sample; the other axes keep none."""
    w = W.suite(name, d=d, ncall=30_000)
    rng = np.random.default_rng(7)
    row = np.cumsum(rng.uniform(0.2, 1.0, w.nb))
    row /= row[-1]
    row[-1] = 1.0
    B = np.tile(row, (d, 1))
    plain = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, nb=w.nb)
    one = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, nb=w.nb, one_dim=True)
    s0, C0, H0, _ = plain.vsample(B, 3, True, hits=True)
    s1, C1, H1, _ = one.vsample(B, 3, True, hits=True)
    assert np.array_equal(s0, s1)
    assert np.array_equal(C1[0], C0[0]) and np.array_equal(H1[0], H0[0])
    assert not C1[1:].any() and not H1[1:].any()
    assert H1[0].sum() == plain.n_samples            # every sample lands in one bin of axis 0
    # no-adjust passes are the same pass
    t0, _, _, _ = plain.vsample(B, 4, False)
    t1, _, _, _ = one.vsample(B, 4, False)
    assert np.array_equal(t0, t1)


def test_first_rebin_spreads_axis0_to_every_axis():
    """One adjusting iteration from the uniform grid: every axis receives
    the rebinning of axis 0's histogram (Lepage's step, pinned separately)."""
    w = W.suite("f2", d=3, ncall=20_000, itmax=1)
    r = _run(w, one_dim=True)
    B0, L0 = oracle.init_grid(1, w.nb, with_lo=True)
    st, Bn = oracle.rebin_axis(r["hist"][0], B0[0], 1.5, L0[0])
    assert st == 0
    for j in range(3):
        assert np.array_equal(r["grid"][j], Bn)
    assert not r["hist"][1:].any()


def test_rows_stay_equal_and_trace_matches_manual_driver():
    """Several adjusting iterations: the grid rows stay equal, and the run
    equals a driver written out here from the pinned pieces (V-Sample with
    the variant's histogram, rebin of axis 0, copy to all axes, weights)."""
    w = W.suite("f5", d=3, ncall=12_000, itmax=4)
    r = _run(w, one_dim=True)
    assert all(np.array_equal(r["grid"][j], r["grid"][0]) for j in range(3))
    pb = oracle.Problem(w.fid, w.params, w.lo, w.hi, w.ncall, nb=w.nb, one_dim=True)
    B, L = oracle.init_grid(3, w.nb, with_lo=True)
    I, V = [], []
    for it in range(w.itmax):
        sums, C, _, _ = pb.vsample(B, it, True, Blo=L)
        I.append(sums[0] / pb.m)
        V.append(sums[1] / pb.m ** 2)
        _, b0, l0 = oracle.rebin_axis(C[0], B[0], 1.5, L[0], with_lo=True)
        B, L = np.tile(b0, (3, 1)), np.tile(l0, (3, 1))
    assert np.array_equal(r["trace_I"], I) and np.array_equal(r["trace_var"], V)
    assert np.array_equal(r["grid"], B)
    est, sig, chi2, _ = oracle.weighted(I, V)
    assert (r["estimate"], r["sigma"], r["chi2_dof"]) == (est, sig, chi2)


@pytest.mark.slow
@pytest.mark.parametrize("name,d", [("f2", 4), ("f4", 5), ("f5", 4), ("f3", 4)])
def test_estimates_match_closed_forms(name, d):
    """The symmetric integrals of the suite (f2, f4, f5) and a non-symmetric
    one (f3: the shared grid adapts poorly, but every estimate stays
    unbiased): within 4 sigma of the closed form."""
    w = W.suite(name, d=d, ncall=60_000, itmax=8, seed=11)
    r = _run(w, one_dim=True)
    exact = CF.exact(w)
    assert r["status"] in (0, 5)
    assert abs(r["estimate"] - exact) <= 4 * r["sigma"], (r["estimate"], exact, r["sigma"])
