"""Accuracy of the library's double-precision log and exp (table-driven,
fixed-point series; used by the FP64 integrands) against 40-digit
references and against CUDA's own functions."""
import math

import mpmath
import numpy as np
import pytest

from paper_2202_01753_gb300 import mcubes

pytestmark = pytest.mark.gpu


def _eval(torch, which, xs):
    d_in = torch.tensor(xs, dtype=torch.float64, device="cuda")
    d_out = torch.empty_like(d_in)
    st = mcubes.lib().mcubes_selftest_fxmath(which, len(xs), d_in.data_ptr(), d_out.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream)
    assert st == mcubes.OK
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


@pytest.fixture(scope="module")
def torch_cuda(gpu_ctx_factory):
    import torch
    return torch


def test_log_accuracy(torch_cuda):
    rng = np.random.default_rng(3)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 3000)), rng.uniform(0.01, 5.0, 3000),
                         1.0 + rng.uniform(-1e-3, 1e-3, 500), [1.0, 2.0, 0.5, 0.05, 1e-300, 1.7e308]])
    got = _eval(torch_cuda, 0, xs)
    cuda = _eval(torch_cuda, 2, xs)
    mpmath.mp.dps = 40
    for x, g, c in zip(xs[::3], got[::3], cuda[::3]):
        ref = mpmath.log(mpmath.mpf(float(x)))
        err = abs(mpmath.mpf(float(g)) - ref)
        assert err <= math.ulp(float(ref)) * 1.01 + 2.0 ** -58, (x, g, float(ref))
    # against CUDA's log: within 2 ulp plus the absolute term everywhere
    tol = 2 * np.spacing(np.abs(cuda)) + 2.0 ** -57
    assert np.all(np.abs(got - cuda) <= tol)
    # outside the fast range it defers to CUDA's log
    special = np.array([0.0, -1.0, np.inf, np.nan, 1e-310])
    g, c = _eval(torch_cuda, 0, special), _eval(torch_cuda, 2, special)
    assert np.array_equal(np.isnan(g), np.isnan(c)) and np.all((g == c) | np.isnan(g))


def test_exp_accuracy(torch_cuda):
    rng = np.random.default_rng(4)
    ys = np.concatenate([rng.uniform(-707.9, 708.9, 3000), rng.uniform(-3, 3, 3000),
                         rng.uniform(-1e-6, 1e-6, 500), [0.0, 1.0, -1.0, 0.0013, -700.0, 700.0]])
    got = _eval(torch_cuda, 1, ys)
    cuda = _eval(torch_cuda, 3, ys)
    mpmath.mp.dps = 40
    for y, g in zip(ys[::3], got[::3]):
        ref = mpmath.exp(mpmath.mpf(float(y)))
        assert abs(mpmath.mpf(float(g)) - ref) / ref <= 2.0 ** -52, (y, g, float(ref))
    assert np.all(np.abs(got - cuda) <= 2 * np.spacing(np.abs(cuda)))
    special = np.array([-800.0, 800.0, -np.inf, np.inf, np.nan, 709.5, -745.2,
                        np.nextafter(-745.2, -np.inf), -746.0, -1e5, -1e300, -np.finfo(np.float64).max])
    g, c = _eval(torch_cuda, 1, special), _eval(torch_cuda, 3, special)
    assert np.array_equal(np.isnan(g), np.isnan(c)) and np.all((g == c) | np.isnan(g))
    # below -745.2 the result is +0 exactly (exp(y) < 2^-1075), as libm gives
    assert np.all(g[special < -745.2] == 0.0) and not np.any(np.signbit(g[special < -745.2]))


def test_exp_subnormal_results(torch_cuda):
    """From y = -708 down to -745.2 the results leave the normal range; they
    are assembled with integer rounding: within one unit of their last
    place (2^-1074 once subnormal) of the 40-digit reference and of CUDA's
    exp, never negative."""
    rng = np.random.default_rng(6)
    ys = np.concatenate([rng.uniform(-745.2, -707.5, 3000), np.linspace(-708.5, -708.3, 100),
                         [-708.5, -745.1, -745.13, -745.14, -744.44007192138]])
    got = _eval(torch_cuda, 1, ys)
    cuda = _eval(torch_cuda, 3, ys)
    mpmath.mp.dps = 40
    tiny = 2.0 ** -1074
    for y, g in zip(ys, got):
        ref = mpmath.exp(mpmath.mpf(float(y)))
        assert abs(mpmath.mpf(float(g)) - ref) <= max(ref * mpmath.mpf(2) ** -52, mpmath.mpf(tiny)), (y, g)
    assert np.all(np.abs(got - cuda) <= np.maximum(2 * np.spacing(np.abs(cuda)), tiny))
    assert np.all(got >= 0.0)


def test_cosf_accuracy(torch_cuda):
    """The mixed-precision kernels' cosine against a 40-digit reference and
    CUDA's cosf, on the single-precision values of the inputs."""
    rng = np.random.default_rng(5)
    xs = np.concatenate([rng.uniform(-30, 30, 4000), rng.uniform(-3.2, 3.2, 2000),
                         rng.uniform(-1e6, 1e6, 1000), [0.0, 1e-30, np.pi / 4, np.pi / 2, np.pi, 7e4, -1e5]])
    xs = xs.astype(np.float32).astype(np.float64)
    got = _eval(torch_cuda, 4, xs)
    cuda = _eval(torch_cuda, 5, xs)
    mpmath.mp.dps = 40
    worst = 0.0
    for x, g in zip(xs, got):
        ref = float(mpmath.cos(mpmath.mpf(float(x))))
        worst = max(worst, abs(g - ref))
    assert worst <= 4 * 2.0 ** -24, worst
    assert np.max(np.abs(got - cuda)) <= 4 * 2.0 ** -24
    huge = np.array([5e6, -3e7, 1e30], dtype=np.float32).astype(np.float64)
    g = _eval(torch_cuda, 4, huge)                    # hardware approximation: a value in [-1, 1]
    assert np.all(np.abs(g) <= 1.0)


def test_exp_scaled_accuracy(torch_cuda):
    """exp(-v) times the fixed factor J = (0xD3C21BCECCEDA100 / 2^63) 2^40,
    rounded once (the cosmo6 kernel's integrand times its Jacobian): within
    2^-52 relative where the product is normal (within one unit of the last
    place, 2^-1074, where it is subnormal), +inf beyond the range, +0 where
    exp(-v) alone rounds to +0 (as exp(-v) * J would)."""
    jm, je = 0xD3C21BCECCEDA100, 40
    rng = np.random.default_rng(5)
    vs = np.concatenate([rng.uniform(-705, 708, 3000), rng.uniform(-3, 3, 2000), rng.uniform(708, 745, 500),
                         [0.0, 1.0, -1.0, -680.0, 745.3, 800.0]])
    got = _eval(torch_cuda, 6, vs)
    mpmath.mp.dps = 50
    J = mpmath.mpf(jm) * mpmath.mpf(2) ** (je - 63)
    for v, g in zip(vs, got):
        ref = mpmath.exp(-mpmath.mpf(float(v))) * J
        if v > 745.2:
            assert g == 0.0
        elif ref > mpmath.mpf(2) ** 1024:
            assert g == math.inf, (v, g)
        else:
            tol = max(ref * mpmath.mpf(2) ** -52, mpmath.mpf(2) ** -1074)
            assert abs(mpmath.mpf(float(g)) - ref) <= tol, (v, g, float(ref))

