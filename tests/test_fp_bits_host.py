"""The integer addition of non-negative doubles that the FP64 histograms'
compare-and-swap retries use (csrc/fp_bits.cuh), compiled for the host
(tests/fpbits_host.cpp): its result must equal the IEEE-754 sum (round to
nearest, ties to even) bit for bit -- random operands over the whole
exponent range, operands close in size and far apart, exact ties, carries
into a new binade and out of the largest finite value, subnormals and zero."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2202_01753_gb300", "csrc")


@pytest.fixture(scope="module")
def addhost(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("fpbits") / "fpbits_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, "-o", exe,
                    os.path.join(HERE, "fpbits_host.cpp")], check=True)

    def run(a, b):
        inp = "\n".join(f"{float(x).hex()} {float(y).hex()}" for x, y in zip(a, b))
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
        return np.array([int(v, 16) for v in out[0::2]], dtype=np.uint64), \
            np.array([int(v, 16) for v in out[1::2]], dtype=np.uint64)
    return run


def _from_bits(u):
    return np.asarray(u, dtype=np.uint64).view(np.float64)


def test_random_operands_every_exponent_gap(addhost):
    rng = np.random.default_rng(7)
    n = 20000
    a = np.exp(rng.uniform(-700, 700, n))
    b = a * np.exp(-rng.uniform(0, 45, n))                  # gaps of 0 to ~65 binades
    got, ref = addhost(a, b)
    assert np.array_equal(got, ref)
    got, ref = addhost(b, a)                                # operand order does not matter
    assert np.array_equal(got, ref)


def test_close_operands_ties_and_carries(addhost):
    rng = np.random.default_rng(8)
    base = (rng.integers(1, 2046, 5000).astype(np.uint64) << np.uint64(52)) | \
        rng.integers(0, 1 << 52, 5000, dtype=np.uint64)
    a = _from_bits(base)
    # b one binade below to 56 binades below with low bits forming exact halves
    k = rng.integers(1, 57, 5000).astype(np.uint64)
    shift = k << np.uint64(52)
    b = _from_bits(np.where(base > shift, base - shift, base & np.uint64((1 << 52) - 1)))
    ties = a * 2.0 ** -53                                   # exactly half an ulp of a
    equal = a                                               # a + a: carry into the next binade
    got, ref = addhost(np.concatenate([a, a, a]), np.concatenate([b, ties, equal]))
    assert np.array_equal(got, ref)


def test_subnormals_zero_and_overflow(addhost):
    rng = np.random.default_rng(9)
    sub = _from_bits(rng.integers(0, 1 << 52, 4000, dtype=np.uint64))       # subnormals
    tiny = _from_bits(rng.integers(1 << 52, 3 << 52, 4000, dtype=np.uint64))  # the smallest normals
    big = np.finfo(np.float64).max
    a = np.concatenate([sub, sub, tiny, [0.0, 0.0, 5.0, big, big, big * 0.75]])
    b = np.concatenate([sub[::-1], tiny, sub, [0.0, 3.0, 0.0, big, 1e292, big * 0.5]])
    with np.errstate(over="ignore"):
        got, ref = addhost(a, b)
    assert np.array_equal(got, ref)
