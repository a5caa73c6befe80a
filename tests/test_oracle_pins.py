"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each group pins one oracle function to something independent of it: a
library routine that computes the same textbook quantity (torch float64 on
CPU), a closed form, an invariant of the mathematics, or a 50-digit brute
force (mpmath) on tiny rows.  The groups are chosen so that a plausible slip
in the oracle (a dropped gamma/beta, a wrong sign, unbiased variance, eps in
the wrong place, a missing max shift, a wrong exponent bias or rounding mode)
fails at least one of them.
"""
import math

import mpmath
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O

mpmath.mp.dps = 50


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- formats
def test_bf16_decode_all_codes_match_library():
    codes = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ours = O.bf16_to_double(codes)
    ref = torch.from_numpy(codes.view(np.int16).copy()).view(torch.bfloat16).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])


def test_e4m3_decode_all_codes_match_library():
    codes = np.arange(256, dtype=np.uint16).astype(np.uint8)
    ours = O.e4m3_to_double(codes)
    ref = torch.from_numpy(codes.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(ours), nan)
    assert np.array_equal(ours[~nan], ref[~nan])
    assert O.e4m3_to_double(np.array([0x7E], dtype=np.uint8))[0] == 448.0


def test_bf16_encode_rne_matches_library_on_fp32_values():
    r = _rng(1)
    v = (r.standard_normal(20000) * np.exp(r.uniform(-40, 40, 20000))).astype(np.float32)
    # exact ties: fp32 values whose low 16 bits are 0x8000 (half-way between bf16 codes)
    bits = r.integers(0, 2**7, 2000, dtype=np.uint32) << 16 | 0x8000      # 7 kept fraction bits
    bits |= (r.integers(1, 250, 2000, dtype=np.uint32) << 23)              # finite exponent
    bits |= (r.integers(0, 2, 2000, dtype=np.uint32) << 31)                # sign
    ties = bits.view(np.float32)
    sub = (r.standard_normal(2000) * 1e-39).astype(np.float32)   # fp32 subnormals
    vals = np.concatenate([v, ties, sub, np.float32([0.0, -0.0, 3.3895314e38])])
    ours = O.double_to_bf16(vals.astype(np.float64))
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, ref)


def test_e4m3_encode_rne_and_saturation():
    r = _rng(2)
    v = np.clip(r.standard_normal(20000) * np.exp(r.uniform(-9, 6, 20000)), -448, 448).astype(np.float32)
    # exact ties between neighbouring e4m3 values
    grid = O.e4m3_to_double(np.arange(0, 0x7E, dtype=np.uint8))
    mids = ((grid[1:] + grid[:-1]) / 2).astype(np.float32)
    vals = np.concatenate([v, mids, -mids])
    ours = O.double_to_e4m3(vals.astype(np.float64))
    ref = torch.from_numpy(vals).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(ours, ref)
    # saturating behaviour (satfinite): everything beyond the largest finite
    # value maps to +-448, including what would round up to 480.
    sat = O.double_to_e4m3(np.array([448.0, 463.9, 464.0, 500.0, 1e30, -1e30, -470.0]))
    assert list(sat) == [0x7E, 0x7E, 0x7E, 0x7E, 0x7E, 0xFE, 0xFE]
    # subnormal quantum is 2^-9, smallest subnormal code 0x01
    assert O.double_to_e4m3(np.array([2.0 ** -9]))[0] == 0x01
    assert O.double_to_e4m3(np.array([2.0 ** -10]))[0] == 0x00          # tie -> even (0)
    assert O.double_to_e4m3(np.array([1.5 * 2.0 ** -9]))[0] == 0x02     # tie -> even (2)


# ---------------------------------------------------------------- softmax
@pytest.mark.parametrize("n", [1, 2, 17, 1000, 4099])
def test_softmax_matches_library(n):
    x = _rng(n).standard_normal((3, n)) * 3
    y = O.softmax(x)
    ref = torch.softmax(torch.from_numpy(x), dim=1).numpy()
    assert np.max(np.abs(y - ref) / ref) < 1e-13
    assert np.allclose(y.sum(axis=1), 1.0, rtol=0, atol=1e-14)


def test_softmax_closed_forms():
    n = 1024
    assert np.all(O.softmax(np.full((1, n), 7.25)) == 1.0 / n)          # constant row
    x = np.zeros((1, n)); x[0, 5] = 200.0                                 # one-hot, large T
    y = O.softmax(x)
    assert y[0, 5] == pytest.approx(1.0, abs=1e-80) and y[0, 0] == pytest.approx(math.exp(-200), rel=1e-12)
    # two-value row: k copies of a, n-k copies of b
    a, b, k = 1.5, -0.75, 300
    x = np.concatenate([np.full(k, a), np.full(n - k, b)])[None, :]
    den = k * math.exp(a) + (n - k) * math.exp(b)
    y = O.softmax(x)
    assert y[0, 0] == pytest.approx(math.exp(a) / den, rel=1e-14)
    assert y[0, -1] == pytest.approx(math.exp(b) / den, rel=1e-14)
    # no overflow for large logits (needs the max shift)
    big = O.softmax(np.array([[1000.0, 999.0, 998.0]]))
    e = np.exp([0.0, -1.0, -2.0]); e /= e.sum()
    assert np.allclose(big[0], e, rtol=1e-14, atol=0)


def test_softmax_shift_invariance():
    x = _rng(3).standard_normal((4, 333))
    y0 = O.softmax(x)
    y1 = O.softmax(x + 64.0)
    assert np.max(np.abs(y1 - y0) / y0) < 1e-12


# ---------------------------------------------------------------- log-sum-exp
@pytest.mark.parametrize("n", [1, 3, 4096])
def test_lse_matches_library(n):
    x = _rng(10 + n).standard_normal((5, n)) * 3
    ref = torch.logsumexp(torch.from_numpy(x), dim=1).numpy()
    assert np.allclose(O.logsumexp(x), ref, rtol=1e-14, atol=0)


def test_lse_closed_forms_and_softmax_relation():
    n = 777
    assert O.logsumexp(np.full((1, n), -3.5))[0] == pytest.approx(-3.5 + math.log(n), rel=1e-15)
    x = _rng(4).standard_normal((2, n))
    l0 = O.logsumexp(x)
    assert np.allclose(O.logsumexp(x + 10.0), l0 + 10.0, rtol=1e-14)
    y = O.softmax(x)
    assert np.allclose(y, np.exp(x - l0[:, None]), rtol=1e-13)


# ---------------------------------------------------------------- layernorm
def test_layernorm_matches_library_with_affine():
    n = 2048
    x = _rng(5).standard_normal((3, n)) * 2 + 0.5
    g = 1 + 0.1 * _rng(6).standard_normal(n)
    b = 0.1 * _rng(7).standard_normal(n)
    y = O.layernorm(x, g, b, eps=1e-5)
    ref = F.layer_norm(torch.from_numpy(x), (n,), torch.from_numpy(g), torch.from_numpy(b), eps=1e-5).numpy()
    assert np.max(np.abs(y - ref)) < 1e-12


def test_layernorm_moments_and_closed_form():
    n = 4096
    x = _rng(8).standard_normal((2, n)) * 3
    eps = 1e-5
    y = O.layernorm(x, eps=eps)
    var = x.var(axis=1)                       # numpy's default is the biased variance
    assert np.allclose(y.mean(axis=1), 0.0, atol=1e-14)
    assert np.allclose(y.var(axis=1), var / (var + eps), rtol=1e-12)
    a = 2.5                                   # +-a alternating -> +-a / sqrt(a^2 + eps)
    alt = np.tile([a, -a], n // 2)[None, :]
    ya = O.layernorm(alt, eps=eps)
    assert np.allclose(ya[0], np.tile([1, -1], n // 2) * a / math.sqrt(a * a + eps), rtol=1e-14)


def test_layernorm_offset_mean_no_cancellation():
    n = 8192
    z = _rng(9).standard_normal((1, n))
    y = O.layernorm(1e4 + z, eps=0.0)
    ref = F.layer_norm(torch.from_numpy(z), (n,), eps=0.0).numpy()
    assert np.max(np.abs(y - ref)) < 1e-9


# ---------------------------------------------------------------- rmsnorm
def test_rmsnorm_matches_library():
    n = 3000
    x = _rng(11).standard_normal((3, n)) * 4
    g = 1 + 0.1 * _rng(12).standard_normal(n)
    y = O.rmsnorm(x, g, eps=1e-6)
    ref = F.rms_norm(torch.from_numpy(x), (n,), torch.from_numpy(g), eps=1e-6).numpy()
    assert np.max(np.abs(y - ref)) < 1e-12


def test_rmsnorm_scale_invariance_and_constant_row():
    x = _rng(13).standard_normal((2, 1001))
    y0 = O.rmsnorm(x, eps=0.0)
    assert np.array_equal(O.rmsnorm(x * 2.0 ** 7, eps=0.0), y0)
    assert np.array_equal(O.rmsnorm(x * 2.0 ** -9, eps=0.0), y0)
    g = 1 + 0.1 * _rng(14).standard_normal(64)
    assert np.allclose(O.rmsnorm(np.full((1, 64), -3.0), g, eps=0.0)[0], -g, rtol=1e-15)


# ---------------------------------------------------------------- brute force
def _mp_ops(row, gamma, beta, eps_ln, eps_rms):
    xs = [mpmath.mpf(float(v)) for v in row]
    n = len(xs)
    m = max(xs)
    S = mpmath.fsum(mpmath.exp(v - m) for v in xs)
    sm = [mpmath.exp(v - m) / S for v in xs]
    lse = m + mpmath.log(S)
    mu = mpmath.fsum(xs) / n
    var = mpmath.fsum((v - mu) ** 2 for v in xs) / n
    ln = [(v - mu) / mpmath.sqrt(var + eps_ln) * mpmath.mpf(float(g)) + mpmath.mpf(float(b))
          for v, g, b in zip(xs, gamma, beta)]
    ms = mpmath.fsum(v * v for v in xs) / n
    rms = [v / mpmath.sqrt(ms + eps_rms) * mpmath.mpf(float(g)) for v, g in zip(xs, gamma)]
    return sm, lse, ln, rms


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_all_ops_against_50_digit_brute_force(n):
    r = _rng(100 + n)
    x = r.standard_normal((1, n)) * 5
    g = 1 + 0.1 * r.standard_normal(n)
    b = 0.1 * r.standard_normal(n)
    sm, lse, ln, rms = _mp_ops(x[0], g, b, 1e-5, 1e-6)
    assert np.allclose(O.softmax(x)[0], [float(v) for v in sm], rtol=1e-15, atol=0)
    assert O.logsumexp(x)[0] == pytest.approx(float(lse), rel=1e-15)
    assert np.allclose(O.layernorm(x, g, b, 1e-5)[0], [float(v) for v in ln], rtol=1e-13, atol=1e-15)
    assert np.allclose(O.rmsnorm(x, g, 1e-6)[0], [float(v) for v in rms], rtol=1e-14, atol=0)


# ---------------------------------------------------------------- batch driver
def test_run_decodes_inputs_exactly():
    r = _rng(15)
    x = torch.from_numpy(r.standard_normal((4, 37)).astype(np.float32) * 3)
    xb = x.to(torch.bfloat16)
    y64, _, _ = O.run(O.SOFTMAX, O.BF16, xb.view(torch.int16).numpy(), 4, 37)
    assert np.allclose(y64, O.softmax(xb.to(torch.float64).numpy()), rtol=1e-15, atol=0)
    amax = x.abs().amax(dim=1)
    s = amax / 448
    q = (x / s[:, None]).clamp(-448, 448).to(torch.float8_e4m3fn)
    y64, _, _ = O.run(O.LOGSUMEXP, O.E4M3, q.view(torch.uint8).numpy(), 4, 37, in_scale=s.numpy())
    xdec = q.to(torch.float64).numpy() * s.double().numpy()[:, None]
    assert np.allclose(y64, O.logsumexp(xdec), rtol=1e-15)


def test_run_fp8_output_scale_and_codes():
    r = _rng(16)
    x = r.standard_normal((3, 500)).astype(np.float32) * 3
    y64, enc, osc = O.run(O.SOFTMAX, O.F32, x, 3, 500, out_dtype=O.E4M3, want_encoded=True)
    S = np.exp(x.astype(np.float64) - x.max(axis=1, keepdims=True)).sum(axis=1)
    assert np.allclose(osc, 1.0 / (448.0 * S), rtol=1e-7)        # closed form amax = 1/S
    dec = O.e4m3_to_double(enc) * osc.astype(np.float64)[:, None]
    # within one E4M3 quantum of the scaled value (normal range quantum 2^(e-3))
    t = np.abs(y64) / osc[:, None]
    ulp = np.exp2(np.maximum(np.floor(np.log2(np.maximum(t, 2.0 ** -30))), -6) - 3) * osc[:, None]
    assert np.all(np.abs(dec - y64) <= 0.5 * ulp * (1 + 1e-6))
    assert np.all(enc.max(axis=1) == 0x7E)                          # the max element hits 448
    # BF16 output: RNE of the exact value
    y64b, encb, _ = O.run(O.RMSNORM, O.F32, x, 3, 500, out_dtype=O.BF16, want_encoded=True)
    assert np.array_equal(encb, O.double_to_bf16(y64b))
    # layernorm of a constant row is all zeros: scale 1, codes 0
    c = np.full((1, 64), 2.0, dtype=np.float32)
    _, encc, oscc = O.run(O.LAYERNORM, O.F32, c, 1, 64, out_dtype=O.E4M3, want_encoded=True)
    assert oscc[0] == 1.0 and np.all(encc == 0)


def test_run_rejects_bad_arguments():
    with pytest.raises(ValueError):
        O.run(O.SOFTMAX, O.F32, np.zeros((1, 1), np.float32), 1, 0)
