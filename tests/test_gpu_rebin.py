"""The device's Adjust-Bin-Bounds (exact Q100 integer cumulative weights,
edges in double-double) against the oracle's (double-double cumulative
weights) on chosen histograms: smooth and rough ones, long runs of empty
bins, a single spike, a dynamic range of 1e-300..1e300, the smallest and
largest bin counts, several compression exponents, a grid already adapted,
and the degenerate cases (all-zero: unchanged; non-finite: ENONFINITE).
Both sides place every edge to ~1e-16 of the unit interval; the test holds
them to 1e-14."""
import numpy as np
import pytest

import oracle
from paper_2202_01753_gb300 import mcubes

pytestmark = pytest.mark.gpu

ATOL = 1e-14


@pytest.fixture(scope="module")
def torch_cuda(gpu_ctx_factory):
    import torch
    return torch


def _device_rebin(torch, C, B, L, alpha):
    dC = torch.tensor(C, dtype=torch.float64, device="cuda")
    dB = torch.tensor(B, dtype=torch.float64, device="cuda")
    dL = torch.tensor(L, dtype=torch.float64, device="cuda")
    st = mcubes.lib().mcubes_selftest_rebin(len(C), float(alpha), dC.data_ptr(), dB.data_ptr(), dL.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    return st, dB.cpu().numpy(), dL.cpu().numpy()


def _uniform(nb):
    B, L = oracle.init_grid(1, nb, with_lo=True)
    return B[0], L[0]


def _cases():
    rng = np.random.default_rng(31)
    nb = 500
    yield "smooth", np.exp(-((np.arange(nb) - 200.0) / 40.0) ** 2) + 1e-3, 1.5, nb
    yield "rough", rng.exponential(1.0, nb), 1.5, nb
    c = rng.exponential(1.0, nb)
    c[rng.random(nb) < 0.9] = 0.0
    yield "mostly_empty", c, 1.5, nb
    c = np.zeros(nb)
    c[317] = 5.0
    yield "single_spike", c, 1.5, nb
    yield "dynamic_range", 10.0 ** rng.uniform(-300, 300, nb), 1.5, nb
    yield "nb2", np.array([3.0, 1.0]), 1.5, 2
    yield "nb3_edge_spike", np.array([0.0, 0.0, 7.0]), 1.5, 3
    yield "nb1024", rng.exponential(1.0, 1024), 1.5, 1024
    for a in (0.5, 1.0, 2.0):
        yield f"alpha{a}", rng.exponential(1.0, nb) ** 3, a, nb


@pytest.mark.parametrize("name,C,alpha,nb", list(_cases()), ids=[c[0] for c in _cases()])
def test_rebin_matches_oracle(torch_cuda, name, C, alpha, nb):
    B, L = _uniform(nb)
    st_o, Bo, Lo = oracle.rebin_axis(C, B, alpha=alpha, Blo=L, with_lo=True)
    st_g, Bg, Lg = _device_rebin(torch_cuda, C, B, L, alpha)
    assert st_o == 0 and st_g == mcubes.OK
    assert Bg[-1] == 1.0 and Lg[-1] == 0.0
    assert np.all(np.diff(Bg) >= 0)
    np.testing.assert_allclose(Bg + Lg, Bo + Lo, rtol=0, atol=ATOL)


def test_rebin_of_an_adapted_grid(torch_cuda):
    """Three rebins in a row from the same histograms: the later ones start
    from non-uniform double-double edges."""
    rng = np.random.default_rng(32)
    nb = 500
    Bo, Lo = _uniform(nb)
    Bg, Lg = Bo.copy(), Lo.copy()
    for _ in range(3):
        C = np.exp(-((np.arange(nb) - 250.0) / 10.0) ** 2) * rng.uniform(0.5, 1.5, nb) + 1e-6
        _, Bo, Lo = oracle.rebin_axis(C, Bo, Blo=Lo, with_lo=True)
        st, Bg, Lg = _device_rebin(torch_cuda, C, Bg, Lg, 1.5)
        assert st == mcubes.OK
        np.testing.assert_allclose(Bg + Lg, Bo + Lo, rtol=0, atol=ATOL)


def test_all_zero_histogram_keeps_the_grid(torch_cuda):
    rng = np.random.default_rng(33)
    B = np.sort(rng.uniform(0, 1, 100))
    B[-1] = 1.0
    L = np.zeros(100)
    st, Bg, Lg = _device_rebin(torch_cuda, np.zeros(100), B, L, 1.5)
    assert st == mcubes.OK
    assert np.array_equal(Bg, B) and np.array_equal(Lg, L)


def test_nonfinite_histogram_is_reported(torch_cuda):
    C = np.ones(50)
    C[7] = np.inf
    B, L = _uniform(50)
    st, _, _ = _device_rebin(torch_cuda, C, B, L, 1.5)
    assert st == mcubes.ENONFINITE
    assert mcubes.lib().mcubes_selftest_rebin(1, 1.5, 0, 0, 0, None) == mcubes.EINVAL
