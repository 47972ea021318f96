"""Pins of the oracle's Weighted-Estimates and Check-Convergence (Alg. 2,
Sec. 5.1): inverse-variance weighting and chi^2 per degree of freedom."""
import numpy as np
import pytest

import oracle


def test_equal_variances_reduce_to_plain_mean():
    I = np.array([1.0, 2.0, 4.0, 7.0])
    est, sig, chi2, conv = oracle.weighted(I, np.full(4, 0.25))
    assert est == pytest.approx(I.mean(), rel=1e-15)
    assert sig == pytest.approx(0.5 / 2.0, rel=1e-15)
    # chi^2/dof = sum (I - mean)^2 / var / (n-1) = sample variance / var
    assert chi2 == pytest.approx(I.var(ddof=1) / 0.25, rel=1e-14)


def test_two_iterations_by_hand():
    # w = (1/4, 1): I = (0.25*1 + 1*3)/1.25 = 2.6, sigma = 1/sqrt(1.25),
    # chi^2 = (1-2.6)^2/4 + (3-2.6)^2/1 = 0.64 + 0.16 = 0.8
    est, sig, chi2, conv = oracle.weighted([1.0, 3.0], [4.0, 1.0])
    assert est == pytest.approx(2.6, rel=1e-15)
    assert sig == pytest.approx(1 / np.sqrt(1.25), rel=1e-15)
    assert chi2 == pytest.approx(0.8, rel=1e-14)


def test_single_iteration_never_converges():
    est, sig, chi2, conv = oracle.weighted([5.0], [1e-20], rel_tol=1.0)
    assert est == 5.0 and chi2 == 0.0 and not conv


def test_convergence_rule():
    I, V = [10.0, 10.0], [0.02, 0.02]  # sigma = 0.1
    assert oracle.weighted(I, V, rel_tol=0.0101)[3]
    assert not oracle.weighted(I, V, rel_tol=0.0099)[3]
    assert oracle.weighted(I, V, rel_tol=0.0, abs_tol=0.1)[3]
    assert not oracle.weighted(I, V, rel_tol=0.0, abs_tol=0.099)[3]


def test_exact_iterations():
    est, sig, chi2, conv = oracle.weighted([3.0, 3.5, 3.0], [1.0, 0.0, 0.0], rel_tol=1e-9)
    assert est == 3.25 and sig == 0.0 and conv


def test_chi2_is_one_on_average():
    # iterations drawn from N(mu, s_i^2): chi^2/dof averages 1
    rng = np.random.default_rng(8)
    vals = []
    for _ in range(2000):
        s = rng.uniform(0.5, 2.0, size=6)
        I = 3.0 + s * rng.standard_normal(6)
        vals.append(oracle.weighted(I, s * s)[2])
    assert np.mean(vals) == pytest.approx(1.0, abs=0.05)
