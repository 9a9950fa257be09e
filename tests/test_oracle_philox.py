"""Oracle pin: Philox4x32-10 sample streams (Salmon et al. SC'11).

Pinned by the generator's published known-answer vectors and by uniformity of the
24-bit uniforms the renderer draws from it.
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_known_answer_vectors():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        got = oracle.philox(ctr, key)
        assert [int(x) for x in got] == expect


def test_uniform_chi_square():
    # 24-bit uniforms u = (r >> 8) * 2^-24 from word 0 over consecutive counters:
    # chi-square over 64 bins must be within the 99.9% band of chi2(63)
    n = 1 << 14
    words = np.array([oracle.philox([i, 3, 0, 0], [12345, 678])[0] for i in range(n)], np.uint64)
    u = (words >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    assert u.min() >= 0.0 and u.max() < 1.0
    hist = np.bincount((u * 64).astype(int), minlength=64)
    e = n / 64
    chi2 = ((hist - e) ** 2 / e).sum()
    assert 30.0 < chi2 < 104.0   # chi2(63): 0.05% and 99.95% quantiles are about 31 and 103


def test_streams_independent():
    # changing one counter word or one key word changes all four output words
    base = oracle.philox([1, 2, 3, 4], [5, 6])
    for k in range(4):
        c = [1, 2, 3, 4]
        c[k] ^= 1
        assert np.all(oracle.philox(c, [5, 6]) != base)
    assert np.all(oracle.philox([1, 2, 3, 4], [5, 7]) != base)
