"""Golden text fixtures (written by tests/golden/make_golden.py from the oracle).

The fixtures guard the oracle against regressions; the closed-form checks
below pin the fixtures themselves: the ramp 4 n1 + n2 is a sum of two
separable terms, so its 2D DCT-II vanishes off row 0 and column 0 and equals
scaled 1D transforms of 0..3 there.
"""

import math
import os

import numpy as np

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    return np.loadtxt(os.path.join(HERE, name))


def dct1_ramp(n):
    return np.array([sum(j * math.cos(math.pi * k * (2 * j + 1) / (2 * n)) for j in range(n))
                     for k in range(n)])


def ramp(n1, n2):
    return (np.arange(n1)[:, None] * n2 + np.arange(n2)[None, :]).astype(np.float64)


def test_dct2d_4x4_fixture_and_closed_form():
    g = load("dct2d_4x4.txt")
    np.testing.assert_allclose(oracle.dct2_2d(ramp(4, 4)), g, atol=1e-12)
    d = dct1_ramp(4)
    expect = np.zeros((4, 4))
    expect[0, 0] = 4 * 4 * 6 + 4 * 6
    expect[1:, 0] = 4 * 4 * d[1:]      # 4 n1 term: N2 * 4 * DCT(0..3)[k1]
    expect[0, 1:] = 4 * d[1:]          # n2 term:  N1 * DCT(0..3)[k2]
    np.testing.assert_allclose(g, expect, atol=1e-12)


def test_idct2d_4x4_fixture_round_trip():
    g = load("idct2d_4x4.txt")
    np.testing.assert_allclose(oracle.idct2_2d(ramp(4, 4)), g, atol=1e-12)
    np.testing.assert_allclose(oracle.dct2_2d(g), ramp(4, 4), atol=1e-12)


def test_dct2d_2x8_checkerboard_fixture():
    g = load("dct2d_2x8.txt")
    x = (-1.0) ** (np.arange(2)[:, None] + np.arange(8)[None, :])
    np.testing.assert_allclose(oracle.dct2_2d(x), g, atol=1e-12)
    # (-1)^n1 over N1 = 2 projects only on k1 = 1 with cos(pi/4) - cos(3pi/4) = sqrt(2)
    assert np.abs(g[0]).max() < 1e-12
    alt = np.array([sum((-1) ** j * math.cos(math.pi * k * (2 * j + 1) / 16) for j in range(8))
                    for k in range(8)])
    np.testing.assert_allclose(g[1], math.sqrt(2) * alt, atol=1e-12)
