"""The kernels' fixed-point log and exp (csrc/fx_math.cuh), compiled for the
host with stand-ins for the device intrinsics (tests/fxmath_host.cpp), against
40-digit references: log within 1 ulp plus 2^-58 absolute, exp within 2^-52
relative (also when scaled by a 64-bit fixed-point factor), and the special
values.  The GPU tests check the same functions on the device against these
bounds and against CUDA's log and exp."""
import math
import os
import shutil
import subprocess

import mpmath
import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_01753_gb300", "csrc")


@pytest.fixture(scope="module")
def fxhost(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fx") / "fxmath_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe, os.path.join(HERE, "fxmath_host.cpp")],
                   check=True)

    def run(xs, scale=None):
        if scale is None:
            lines = [float(x).hex() for x in xs]
        else:
            lines = [f"{float(x).hex()} {int(m)} {int(e)}" for x, (m, e) in zip(xs, scale)]
        out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                             text=True, check=True).stdout.split()
        if scale is not None:
            return np.array([float.fromhex(v) for v in out])
        return (np.array([float.fromhex(v) for v in out[0::2]]),
                np.array([float.fromhex(v) for v in out[1::2]]))
    return run


def _bits(x):
    return int(np.float64(x).view(np.uint64))


def _dbl(b):
    return float(np.uint64(b).view(np.float64))


def test_log_accuracy_host(fxhost):
    rng = np.random.default_rng(21)
    xs = np.concatenate([np.exp(rng.uniform(-700, 700, 4000)), rng.uniform(0.01, 5.0, 4000),
                         1.0 + rng.uniform(-1e-3, 1e-3, 1000)])
    # the ends of every table interval, values next to 1, the extremes of the range
    edges = [_dbl((1023 << 52) | (j << 44) | d) for j in range(256) for d in (0, 1, (1 << 44) - 1)]
    near1 = [_dbl(_bits(1.0) - k) for k in range(1, 40)] + [_dbl(_bits(1.0) + k) for k in range(0, 40)]
    ends = [_dbl(((1023 + e) << 52) | (255 << 44) | ((1 << 44) - 1)) for e in range(-1022, 1024, 7)]
    # the second step's table points (1 + j/256)(1 + k/65536) and their neighbours
    second = [(1 + j / 256) * (1 + k / 65536) for j in range(0, 256, 9) for k in range(0, 256, 11)]
    second = np.concatenate([second, np.nextafter(second, 0), np.nextafter(second, 3)])
    xs = np.concatenate([xs, edges, near1, ends, second, [2.2250738585072014e-308, 1.7976931348623157e308]])
    got, _ = fxhost(xs)
    mpmath.mp.dps = 40
    for x, g in zip(xs, got):
        ref = mpmath.log(mpmath.mpf(float(x)))
        tol = math.ulp(float(ref)) * 1.01 + 2.0 ** -58
        assert abs(mpmath.mpf(float(g)) - ref) <= tol, (x, g, float(ref))
    assert got[list(xs).index(1.0)] == 0.0


def test_exp_accuracy_host(fxhost):
    rng = np.random.default_rng(22)
    ys = np.concatenate([rng.uniform(-708.9, 707.9, 4000), rng.uniform(-3, 3, 4000),
                         rng.uniform(-1e-6, 1e-6, 500), [0.0, 1.0, -1.0, -700.0, 700.0]])
    # arguments at and next to multiples of ln2/256 and halfway between them,
    # where the reduction picks n
    steps = np.array([n * math.log(2) / 256 for n in range(-2000, 2000, 7)] +
                     [(n + 0.5) * math.log(2) / 256 for n in range(-2000, 2000, 7)])
    ys = np.concatenate([ys, steps, np.nextafter(steps, np.inf), np.nextafter(steps, -np.inf)])
    _, got = fxhost(ys)      # fx_exp(-y)
    mpmath.mp.dps = 40
    for y, g in zip(ys, got):
        ref = mpmath.exp(-mpmath.mpf(float(y)))
        assert abs(mpmath.mpf(float(g)) - ref) / ref <= 2.0 ** -52, (y, g, float(ref))
    # exp(y) for y < -745.2 (to -inf) is +0 exactly
    _, z = fxhost([745.3, 800.0, 1e5, 1e300, math.inf])
    assert np.all(z == 0.0) and not np.any(np.signbit(z))


def test_exp_subnormal_results_host(fxhost):
    """exp(y) for y from -708 down to -745.2, where the result leaves the
    normal range: assembled with integer rounding, within one unit of the
    last place of the result (2^-1074 once subnormal), +0 below 2^-1075."""
    rng = np.random.default_rng(23)
    ys = np.concatenate([rng.uniform(707.5, 745.2, 6000), np.linspace(708.3, 708.5, 200),
                         np.linspace(744.4, 745.2, 200),
                         [708.0, 708.3964185322641, 708.4, 744.4400719213812, 745.1332191019411, 745.13, 745.2]])
    _, got = fxhost(ys)      # fx_exp(-y)
    mpmath.mp.dps = 40
    tiny = mpmath.mpf(2) ** -1074
    for y, g in zip(ys, got):
        ref = mpmath.exp(-mpmath.mpf(float(y)))
        tol = max(ref * mpmath.mpf(2) ** -52, tiny)
        assert abs(mpmath.mpf(float(g)) - ref) <= tol, (y, g, float(ref))
    assert np.all(got >= 0.0)


def test_exp_scaled_host(fxhost):
    """exp(-v) (jm / 2^63) 2^je, rounded once (the FP64 kernels' integrand
    exponential times their Jacobian): within 2^-52 relative wherever the
    result is normal, +inf on overflow, and +0 wherever exp(-v) alone rounds
    to +0 (v > 745.2), as the product of the two doubles would be."""
    rng = np.random.default_rng(24)
    vs = np.concatenate([rng.uniform(-705, 708, 4000), rng.uniform(-3, 3, 2000), rng.uniform(708, 745, 1000),
                         rng.uniform(-1e-6, 1e-6, 200), [0.0, 1.0, -1.0]])
    jm = rng.integers(2 ** 63, 2 ** 64 - 1, len(vs), dtype=np.uint64, endpoint=True)
    jm[:8] = [2 ** 63, 2 ** 64 - 1] * 4
    je = rng.integers(-80, 81, len(vs))
    got = fxhost(vs, scale=list(zip(jm, je)))
    mpmath.mp.dps = 50
    checked = 0
    for v, m, e, g in zip(vs, jm, je, got):
        ref = mpmath.exp(-mpmath.mpf(float(v))) * int(m) * mpmath.mpf(2) ** (int(e) - 63)
        if ref > mpmath.mpf(2) ** 1024:
            assert g == math.inf, (v, m, e, g)
        elif ref >= mpmath.mpf(2) ** -1022 and v < 708.39:
            assert abs(mpmath.mpf(float(g)) - ref) / ref <= 2.0 ** -52, (v, m, e, g, float(ref))
            checked += 1
        else:  # exp(-v) subnormal: the product is exact to the last place of the result
            assert abs(mpmath.mpf(float(g)) - ref) <= max(ref * mpmath.mpf(2) ** -52, mpmath.mpf(2) ** -1074)
    assert checked > 5000
    z = fxhost([745.3, 800.0, math.inf], scale=[(2 ** 64 - 1, 80)] * 3)
    assert np.all(z == 0.0) and not np.any(np.signbit(z))


def test_tables_header_is_generated():
    """csrc/fx_tables.h is exactly what gen_fx_tables.py computes from the
    constants' definitions (60-digit arithmetic, rounded once): no entry is
    edited by hand."""
    from paper_2202_01753_gb300 import gen_fx_tables as G
    with open(G.OUT) as f:
        assert f.read() == G.render()
