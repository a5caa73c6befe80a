"""Pins of the oracle's row-wise int8 quantisation (the "row-wise int8
quantization" workload): numpy float32 arithmetic (IEEE division, rint ties
to even) as the library routine for the same definition, the error bound of
the dequantised values, exact cases (the amax element, ties, all-zero rows),
and the exact invariance under scaling by powers of two."""
import numpy as np
import pytest

import oracle as O


def _numpy_quant(x):
    x = np.asarray(x, dtype=np.float32)
    amax = np.abs(x).max(axis=1)
    s = np.where(amax > 0, (amax / np.float32(127)).astype(np.float32), np.float32(1))
    q = np.clip(np.rint(x / s[:, None]), -127, 127).astype(np.int8)
    return q, s


def test_matches_numpy_float32_arithmetic():
    r = np.random.default_rng(1)
    x = (r.standard_normal((64, 1000)) * np.exp(r.uniform(-20, 20, (64, 1)))).astype(np.float32)
    x[::7, ::13] = 50.0 * np.sign(x[::7, ::13])        # outliers set the scale
    q, s = O.quant_int8(x)
    qn, sn = _numpy_quant(x)
    assert np.array_equal(s, sn)
    assert np.array_equal(q, qn)


def test_dequantisation_error_bound_and_the_amax_element():
    r = np.random.default_rng(2)
    x = r.standard_normal((20, 513)).astype(np.float32) * 3
    q, s = O.quant_int8(x)
    err = np.abs(q.astype(np.float64) * s[:, None] - x)
    assert (err <= 0.5 * s[:, None] * (1 + 1e-6) + 1e-30).all()
    i = np.abs(x).argmax(axis=1)
    assert np.array_equal(np.abs(q[np.arange(20), i]), np.full(20, 127, dtype=np.int8))
    assert np.abs(q).max() <= 127 and q.min() >= -127


def test_exact_cases():
    # x = s * (k + 1/2) for exactly representable s: ties go to the even integer
    s = np.float32(0.5)
    x = np.array([[63.5, 0.25, 0.75, -0.25, -0.75, 1.25, 0.0, 2.0]], dtype=np.float32)  # amax 63.5 -> s = 0.5
    q, sc = O.quant_int8(x)
    assert sc[0] == s
    assert q[0].tolist() == [127, 0, 2, 0, -2, 2, 0, 4]
    z, sz = O.quant_int8(np.zeros((2, 9), dtype=np.float32))
    assert (z == 0).all() and (sz == 1).all()


@pytest.mark.parametrize("k", [-30, -3, 5, 40])
def test_power_of_two_scaling_is_exact(k):
    r = np.random.default_rng(3)
    x = r.standard_normal((8, 300)).astype(np.float32)
    q, s = O.quant_int8(x)
    q2, s2 = O.quant_int8((x * np.float32(2.0 ** k)).astype(np.float32))
    assert np.array_equal(q, q2)
    assert np.array_equal(s2, (s * np.float32(2.0 ** k)).astype(np.float32))
