"""The retry rule for unconverged integrals (paper_2202_01753_gb300.retry,
the server's rule written for host loops): the fixed form, and the sized
form whose calls follow sigma ~ (calls x iterations)^-1/2."""
import math

from paper_2202_01753_gb300.retry import retry_ncall


def test_fixed_factor_stops_at_the_cap():
    assert retry_ncall(100_000, 1.0, 1.0, 1e-4, 0.0, 4.0, 0.0, 10 ** 6) == 400_000
    assert retry_ncall(400_000, 1.0, 1.0, 1e-4, 0.0, 4.0, 0.0, 10 ** 6) == 400_000   # 1.6e6 > cap: none


def test_sized_factor_follows_sigma_over_tau():
    # sigma = 3 tau: 2 x 9 = 18 times the calls
    assert retry_ncall(100_000, 2.0, 3 * 2e-4, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 1_800_000
    # at the tolerance: 2 x 1^2, the smallest factor; just below it, still the smallest
    assert retry_ncall(100_000, 1.0, 1e-4, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 200_000
    assert retry_ncall(100_000, 1.0, 0.5e-4, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 200_000
    assert retry_ncall(100_000, 1.0, 1.01e-4, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 204_020
    # far above: the largest factor; the absolute tolerance counts when larger
    assert retry_ncall(100_000, 1.0, 1.0, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 6_400_000
    assert retry_ncall(100_000, 1.0, 2e-3, 1e-4, 1e-3, 2.0, 64.0, 10 ** 9) == 800_000


def test_sized_factor_degenerate_tolerance_and_cap():
    assert retry_ncall(100_000, 0.0, 1.0, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 6_400_000   # tau = 0
    assert retry_ncall(100_000, 1.0, math.inf, 1e-4, 0.0, 2.0, 64.0, 10 ** 9) == 6_400_000
    assert retry_ncall(100_000, 1.0, 1.0, 1e-4, 0.0, 2.0, 64.0, 2_000_000) == 2_000_000
