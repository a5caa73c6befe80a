"""Pins of the oracle's negative-control ops (the screening rule's scan and
stencil cases, Sec. III-D and IV-C): exact prefix sums of integers and of
dyadic values, the first difference of a scan, exact rational prefix sums of
random doubles on short rows, numpy's cumsum and convolve as library routines
for the same definitions, the stencil of a delta (the weights) and of a
constant row (interior sum of the weights, zero-padded ends)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def test_scan_of_ones_and_integers_is_exact():
    y = O.scan(np.ones((2, 1000)))
    assert np.array_equal(y[0], np.arange(1, 1001, dtype=np.float64))
    r = np.random.default_rng(1)
    x = r.integers(-1000, 1000, (5, 777)).astype(np.float64)
    y = O.scan(x)
    assert np.array_equal(y, np.cumsum(x, axis=1))
    assert np.array_equal(np.diff(y, axis=1, prepend=0.0), x)   # the first difference recovers x


def test_scan_is_the_exact_rational_prefix_sum_within_an_ulp():
    r = np.random.default_rng(2)
    x = r.standard_normal((3, 64)) * np.exp(r.uniform(-20, 20, (3, 64)))
    y = O.scan(x)
    for i in range(3):
        acc = Fraction(0)
        for j in range(64):
            acc += Fraction(x[i, j])
            exact = float(acc)
            assert abs(y[i, j] - exact) <= np.spacing(abs(exact)) + 1e-300


def test_scan_matches_numpy_cumsum():
    r = np.random.default_rng(3)
    x = r.standard_normal((4, 5000))
    np.testing.assert_allclose(O.scan(x), np.cumsum(x, axis=1), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("w", [[0.25, 0.5, 0.25], [-1.0, 0.0, 1.0], [0.1, -0.2, 0.4, -0.2, 0.1]])
def test_stencil_matches_numpy_convolve(w):
    r = np.random.default_rng(4)
    x = r.standard_normal((3, 301))
    y = O.stencil(x, w)
    for i in range(3):  # y_i = sum_k w[k + r] x_{i+k}: a convolution with the reversed weights, same size
        np.testing.assert_allclose(y[i], np.convolve(x[i], np.asarray(w)[::-1], mode="same"), rtol=1e-13, atol=1e-13)


def test_stencil_of_a_delta_and_of_a_constant_row():
    w = np.array([0.1, -0.2, 0.4, -0.2, 0.1])
    x = np.zeros((1, 21))
    x[0, 10] = 1.0
    y = O.stencil(x, w)[0]
    assert np.array_equal(y[8:13], w[::-1]) and not y[:8].any() and not y[13:].any()
    c = O.stencil(np.full((1, 50), 3.0), w)[0]
    assert np.allclose(c[2:-2], 3.0 * w.sum(), rtol=0, atol=1e-15)
    assert c[0] == pytest.approx(3.0 * w[2:].sum()) and c[-1] == pytest.approx(3.0 * w[:3].sum())
