"""Pins of the oracle's random stream: Philox4x32-10 known answers and the
statistics of the words the sampler consumes."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_sample_words_layout():
    # word j of a sample is word j mod 4 of the block with counter (s, cube, it, j div 4)
    seed = 0x0123456789ABCDEF
    key = [seed & 0xFFFFFFFF, seed >> 32]
    w = oracle.sample_words(seed, it=7, cube=12345, s=3, d=10)
    for b in range(3):
        blk = oracle.philox4x32_10([3, 12345, 7, b], key)
        for q in range(4):
            if 4 * b + q < 10:
                assert w[4 * b + q] == blk[q]


def test_words_are_uniform():
    # 20000 samples x 4 axes: moments and a chi^2 test on 64 equal cells
    words = np.array([oracle.sample_words(11, 0, c, s, 4) for c in range(2000) for s in range(10)],
                     dtype=np.float64)
    u = (words + 0.5) / 2.0 ** 32
    assert abs(u.mean() - 0.5) < 5 * np.sqrt(1 / 12 / u.size)
    assert abs(u.var() - 1 / 12) < 5 * np.sqrt(1 / 180 / u.size)
    for j in range(4):
        counts = np.bincount((u[:, j] * 64).astype(int), minlength=64)
        assert stats.chisquare(counts).pvalue > 1e-4
    # axes are uncorrelated
    cc = np.corrcoef(u.T)
    assert np.max(np.abs(cc - np.eye(4))) < 5 / np.sqrt(u.shape[0])
