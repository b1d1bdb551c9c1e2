"""Pins of the oracle's primitives against closed forms and statistics.

The integer distance threshold is pinned against exact rational arithmetic,
the probability threshold against its closed form, and Philox4x32-10 against
statistical properties of a keyed bijective generator (the bit-exact
comparison with NVIDIA's cuRAND Philox lives in the GPU tests).
"""

from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("d", [0.0, 0.3, 0.5, 0.6, 1.0, 1.1, 1.3, 2.5, 3.0, 7.25, 1e-7, 123.456])
def test_r2_is_exact_floor_of_square(d):
    # floor((d * 2^20)^2) computed with exact rationals from the double d
    exact = (Fraction(d) * (1 << 20)) ** 2
    assert O.r2(d) == exact.numerator // exact.denominator


def test_r2_closed_forms():
    assert O.r2(1.0) == 1 << 40
    assert O.r2(0.5) == 1 << 38
    assert O.r2(3.0) == 9 << 40
    # the double nearest 1.1 lies above 11/10; its square still floors to 121 * 2^40 / 100
    assert O.r2(1.1) == (121 << 40) // 100
    assert O.r2(-1.0) == 0


@pytest.mark.parametrize("p", [0.0, 1e-12, 0.05, 0.1, 0.3, 0.5, 0.9, 0.999999, 1.0, 1.5, -0.2])
def test_threshold_closed_form(p):
    if p <= 0:
        want = 0
    elif p >= 1:
        want = 1 << 32
    else:
        f = Fraction(p) * (1 << 32)
        want = f.numerator // f.denominator
    assert O.threshold(p) == want


def _philox_many(n, key, word=0, base=(0, 0, 0, 0)):
    out = np.zeros((n, 4), np.uint64)
    for i in range(n):
        c = list(base)
        c[word] = (c[word] + i) & 0xFFFFFFFF
        out[i] = O.philox(c, key)
    return out


def test_philox_uniform_words():
    # 8000 draws x 4 words: each 32-bit word, split into 16 bins, is uniform
    x = _philox_many(8000, (0x1234, 0xABCD), word=0)
    from scipy.stats import chisquare
    for w in range(4):
        counts = np.bincount((x[:, w] >> 28).astype(np.int64), minlength=16)
        assert chisquare(counts).pvalue > 1e-4


def test_philox_avalanche():
    # flipping any single counter or key bit flips about half the output bits
    rng = np.random.default_rng(5)
    flips = []
    for _ in range(200):
        ctr = [int(v) for v in rng.integers(0, 2**32, 4)]
        key = [int(v) for v in rng.integers(0, 2**32, 2)]
        y0 = O.philox(ctr, key)
        which = int(rng.integers(0, 6 * 32))
        c2, k2 = list(ctr), list(key)
        if which < 128:
            c2[which // 32] ^= 1 << (which % 32)
        else:
            k2[(which - 128) // 32] ^= 1 << (which % 32)
        y1 = O.philox(c2, k2)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(y0, y1)))
    m = np.mean(flips)
    assert 60 < m < 68, m
    assert min(flips) > 30


def test_philox_depends_on_every_input_word():
    base_c, base_k = [1, 2, 3, 4], [5, 6]
    y0 = O.philox(base_c, base_k)
    for w in range(4):
        c = list(base_c)
        c[w] ^= 0x80000000
        assert not np.array_equal(O.philox(c, base_k), y0)
    for w in range(2):
        k = list(base_k)
        k[w] ^= 1
        assert not np.array_equal(O.philox(base_c, k), y0)


def test_bernoulli_frequency_matches_p():
    # u < floor(p 2^32) succeeds with probability p (to 2^-32); the average of
    # two uniforms below p has probability 2 p^2 for p <= 1/2
    n = 20000
    x = _philox_many(n, (77, 88), word=0, base=(0, 9, 1, 2))
    for p in (0.05, 0.5, 0.9):
        T = O.threshold(p)
        k = int(np.sum(x[:, 0] < T))
        sd = np.sqrt(n * p * (1 - p))
        assert abs(k - n * p) < 4.5 * sd, (p, k)
    for p in (0.05, 0.3):
        T = O.threshold(p)
        q = 2 * p * p
        k = int(np.sum(x[:, 0] + x[:, 1] < 2 * T))
        sd = np.sqrt(n * q * (1 - q))
        assert abs(k - n * q) < 4.5 * sd, (p, k)
