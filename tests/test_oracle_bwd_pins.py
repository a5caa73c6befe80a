"""Pins of the oracle's input gradients (softmax, LayerNorm, RMSNorm backward).

Each backward op is the vector-Jacobian product of a forward op, so the pins
differentiate the forward definitions independently of the backward code:
central differences of the FP64 forward oracle, a 50-digit mpmath derivative
of the forward written out here on tiny rows, and torch float64 autograd (a
library routine for the same textbook quantity).  Invariants of the
mathematics (the gradient of a shift- or scale-invariant function is
orthogonal to the invariant direction) and exact special cases catch a
dropped term or a wrong sign; the batch driver is pinned to the row functions
and to the formats' rounding.
"""
import mpmath
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O

mpmath.mp.dps = 50


def _rng(seed):
    return np.random.default_rng(seed)


def _ln_stats(x, eps):
    mean = x.mean(axis=1)
    var = ((x - mean[:, None]) ** 2).mean(axis=1)
    return mean, 1.0 / np.sqrt(var + eps)


def _rms_rstd(x, eps):
    return 1.0 / np.sqrt((x * x).mean(axis=1) + eps)


def _row_case(seed, n, offset=0.0):
    r = _rng(seed)
    x = r.standard_normal((3, n)) * 2.0 + offset
    dy = r.standard_normal((3, n))
    gamma = 1.0 + 0.1 * r.standard_normal(n)
    beta = 0.1 * r.standard_normal(n)
    return x, dy, gamma, beta


def _fd_grad(fwd, x, dy, h=1e-5):
    """Central differences of L(x) = sum_j dy_j fwd(x)_j, row by row."""
    g = np.empty_like(x)
    for k in range(x.shape[1]):
        xp, xm = x.copy(), x.copy()
        xp[:, k] += h
        xm[:, k] -= h
        g[:, k] = ((fwd(xp) - fwd(xm)) * dy).sum(axis=1) / (2 * h)
    return g


@pytest.mark.parametrize("n", [2, 7, 33])
def test_softmax_bwd_matches_finite_differences(n):
    x, dy, _, _ = _row_case(1, n)
    dx = O.softmax_bwd(O.softmax(x), dy)
    fd = _fd_grad(O.softmax, x, dy)
    assert np.abs(dx - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("n", [2, 7, 33])
@pytest.mark.parametrize("offset", [0.0, 1e3])
def test_layernorm_bwd_matches_finite_differences(n, offset):
    x, dy, gamma, beta = _row_case(2, n, offset)
    eps = 1e-5
    mean, rstd = _ln_stats(x, eps)
    dx = O.layernorm_bwd(x, dy, mean, rstd, gamma)
    fd = _fd_grad(lambda v: O.layernorm(v, gamma, beta, eps), x, dy, h=1e-5 * (1 + abs(offset)) ** 0.5)
    assert np.abs(dx - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("n", [2, 7, 33])
def test_rmsnorm_bwd_matches_finite_differences(n):
    x, dy, gamma, _ = _row_case(3, n)
    eps = 1e-6
    dx = O.rmsnorm_bwd(x, dy, _rms_rstd(x, eps), gamma)
    fd = _fd_grad(lambda v: O.rmsnorm(v, gamma, eps), x, dy)
    assert np.abs(dx - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max())


def _mp_vjp(fwd, x, dy):
    """dx_k = d/dt sum_j dy_j fwd(x + t e_k)_j at t = 0, in 50-digit arithmetic."""
    xs = [mpmath.mpf(float(v)) for v in x]
    out = []
    for k in range(len(xs)):
        def f(t, k=k):
            v = list(xs)
            v[k] = v[k] + t
            return mpmath.fsum(mpmath.mpf(float(d)) * y for d, y in zip(dy, fwd(v)))
        out.append(float(mpmath.diff(f, 0)))
    return np.array(out)


def _mp_softmax(v):
    m = max(v)
    e = [mpmath.exp(t - m) for t in v]
    s = mpmath.fsum(e)
    return [t / s for t in e]


def _mp_layernorm(gamma, eps):
    def f(v):
        n = len(v)
        mu = mpmath.fsum(v) / n
        var = mpmath.fsum((t - mu) ** 2 for t in v) / n
        r = 1 / mpmath.sqrt(var + eps)
        return [(t - mu) * r * mpmath.mpf(float(g)) for t, g in zip(v, gamma)]
    return f


def _mp_rmsnorm(gamma, eps):
    def f(v):
        r = 1 / mpmath.sqrt(mpmath.fsum(t * t for t in v) / len(v) + eps)
        return [t * r * mpmath.mpf(float(g)) for t, g in zip(v, gamma)]
    return f


def test_tiny_rows_match_a_50_digit_derivative():
    x, dy, gamma, _ = _row_case(4, 5)
    x, dy = x[:1], dy[:1]
    eps_ln, eps_rms = mpmath.mpf("1e-5"), mpmath.mpf("1e-6")
    sm = O.softmax_bwd(O.softmax(x), dy)[0]
    assert np.allclose(sm, _mp_vjp(_mp_softmax, x[0], dy[0]), rtol=1e-12, atol=1e-14)
    mean, rstd = _ln_stats(x, 1e-5)
    ln = O.layernorm_bwd(x, dy, mean, rstd, gamma)[0]
    assert np.allclose(ln, _mp_vjp(_mp_layernorm(gamma, eps_ln), x[0], dy[0]), rtol=1e-12, atol=1e-13)
    rms = O.rmsnorm_bwd(x, dy, _rms_rstd(x, 1e-6), gamma)[0]
    assert np.allclose(rms, _mp_vjp(_mp_rmsnorm(gamma, eps_rms), x[0], dy[0]), rtol=1e-12, atol=1e-13)


def test_torch_float64_autograd_agrees():
    r = _rng(5)
    n = 300
    x = r.standard_normal((4, n)) * 3.0
    dy = r.standard_normal((4, n))
    gamma = 1.0 + 0.1 * r.standard_normal(n)
    beta = 0.1 * r.standard_normal(n)
    tx = torch.tensor(x, requires_grad=True)
    torch.softmax(tx, dim=1).backward(torch.tensor(dy))
    assert np.allclose(O.softmax_bwd(O.softmax(x), dy), tx.grad.numpy(), rtol=1e-12, atol=1e-15)
    tx = torch.tensor(x, requires_grad=True)
    F.layer_norm(tx, (n,), torch.tensor(gamma), torch.tensor(beta), 1e-5).backward(torch.tensor(dy))
    mean, rstd = _ln_stats(x, 1e-5)
    assert np.allclose(O.layernorm_bwd(x, dy, mean, rstd, gamma), tx.grad.numpy(), rtol=1e-10, atol=1e-12)
    tx = torch.tensor(x, requires_grad=True)
    F.rms_norm(tx, (n,), torch.tensor(gamma), 1e-6).backward(torch.tensor(dy))
    assert np.allclose(O.rmsnorm_bwd(x, dy, _rms_rstd(x, 1e-6), gamma), tx.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_gradients_are_orthogonal_to_the_invariant_directions():
    x, dy, gamma, _ = _row_case(6, 64)
    # softmax is shift invariant: the gradient sums to zero
    dx = O.softmax_bwd(O.softmax(x), dy)
    assert np.abs(dx.sum(axis=1)).max() <= 1e-14
    # layernorm (any eps) is shift invariant: the gradient sums to zero
    mean, rstd = _ln_stats(x, 1e-5)
    dx = O.layernorm_bwd(x, dy, mean, rstd, gamma)
    assert np.abs(dx.sum(axis=1)).max() <= 1e-12
    # with eps > 0 it is not scale invariant: sum_i dx_i xh_i = rstd b (N - sum xh^2), b = sum g xh / N
    xh = (x - mean[:, None]) * rstd[:, None]
    b = (dy * gamma * xh).sum(axis=1) / x.shape[1]
    expect = rstd * b * (x.shape[1] - (xh * xh).sum(axis=1))
    assert np.abs((dx * xh).sum(axis=1) - expect).max() <= 1e-12
    # at eps = 0 it is: sum_i dx_i xh_i = 0
    mean, rstd = _ln_stats(x, 0.0)
    dx = O.layernorm_bwd(x, dy, mean, rstd, gamma)
    xh = (x - mean[:, None]) * rstd[:, None]
    assert np.abs((dx * xh).sum(axis=1)).max() <= 1e-12
    # rmsnorm with eps = 0 is scale invariant: sum_i dx_i x_i = 0
    dx = O.rmsnorm_bwd(x, dy, _rms_rstd(x, 0.0), gamma)
    assert np.abs((dx * x).sum(axis=1)).max() <= 1e-12


def test_special_cases():
    x, dy, gamma, _ = _row_case(7, 40)
    # softmax with a constant upstream gradient: no gradient at all
    assert np.abs(O.softmax_bwd(O.softmax(x), np.full_like(x, 2.5))).max() <= 1e-16
    # layernorm with dy * gamma constant: the gradient vanishes (sum xh = 0)
    mean, rstd = _ln_stats(x, 1e-5)
    dx = O.layernorm_bwd(x, 0.75 / gamma[None, :] * np.ones_like(x), mean, rstd, gamma)
    assert np.abs(dx).max() <= 1e-13
    # rmsnorm at eps = 0 with dy parallel to y: the gradient vanishes (scale invariance)
    rstd = _rms_rstd(x, 0.0)
    y = O.rmsnorm(x, gamma, 0.0)
    dx = O.rmsnorm_bwd(x, 3.0 * y / (gamma * gamma)[None, :], rstd, gamma)
    assert np.abs(dx).max() <= 1e-13
    # gamma = None means gamma = 1
    ones = np.ones(x.shape[1])
    assert np.array_equal(O.layernorm_bwd(x, dy, mean, rstd), O.layernorm_bwd(x, dy, mean, rstd, ones))
    assert np.array_equal(O.rmsnorm_bwd(x, dy, rstd), O.rmsnorm_bwd(x, dy, rstd, ones))


@pytest.mark.parametrize("dtype", [O.F32, O.BF16])
def test_batch_driver_matches_row_functions_and_rounding(dtype):
    r = _rng(8)
    rows, cols, ld = 6, 77, 80
    x = (r.standard_normal((rows, ld)) * 2).astype(np.float32)
    dy = r.standard_normal((rows, ld)).astype(np.float32)
    if dtype == O.BF16:
        xr = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        dyr = torch.from_numpy(dy).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        xd, dyd = O.bf16_to_double(xr), O.bf16_to_double(dyr)
    else:
        xr, dyr, xd, dyd = x, dy, x.astype(np.float64), dy.astype(np.float64)
    xd, dyd = xd[:, :cols], dyd[:, :cols]
    gamma = (1 + 0.1 * r.standard_normal(cols)).astype(np.float32)
    mean, rstd = _ln_stats(xd, 1e-5)
    mean32, rstd32 = mean.astype(np.float32), rstd.astype(np.float32)
    rms32 = _rms_rstd(xd, 1e-6).astype(np.float32)
    y = O.softmax(xd)
    cases = [(O.SOFTMAX, xr, {}, O.softmax_bwd(xd, dyd)),
             (O.LAYERNORM, xr, dict(gamma=gamma, mean=mean32, rstd=rstd32),
              O.layernorm_bwd(xd, dyd, mean32.astype(np.float64), rstd32.astype(np.float64), gamma)),
             (O.RMSNORM, xr, dict(gamma=gamma, rstd=rms32),
              O.rmsnorm_bwd(xd, dyd, rms32.astype(np.float64), gamma))]
    del y
    for op, a, kw, ref in cases:
        dx64, enc = O.run_bwd(op, dtype, a, dyr, rows, cols, ld=ld, want_encoded=True, **kw)
        assert np.array_equal(dx64, ref)
        if dtype == O.F32:
            assert np.array_equal(enc, ref.astype(np.float32))
        else:
            assert np.array_equal(enc, O.double_to_bf16(ref))


def test_batch_driver_rejects_bad_arguments():
    a = np.zeros((2, 8), dtype=np.float32)
    with pytest.raises(ValueError):
        O.run_bwd(O.LOGSUMEXP, O.F32, a, a, 2, 8)
    with pytest.raises(ValueError):
        O.run_bwd(O.LAYERNORM, O.F32, a, a, 2, 8, rstd=np.ones(2))        # no mean
    with pytest.raises(ValueError):
        O.run_bwd(O.RMSNORM, O.F32, a, a, 2, 8)                           # no rstd
    with pytest.raises(ValueError):
        O.run_bwd(O.SOFTMAX, O.E4M3, a.view(np.uint8), a.view(np.uint8), 2, 8)


# ---------------------------------------------------------------- gradients with respect to the logits
def _xent_loss(z, t):
    """-sum_j t_j log softmax(z)_j per row, through the oracle's log-sum-exp: log y_j = z_j - LSE(z)."""
    return -(t * (z - O.logsumexp(z)[:, None])).sum(axis=1)


@pytest.mark.parametrize("n", [2, 7, 33])
def test_softmax_logits_bwd_matches_finite_differences(n):
    z, dy, _, _ = _row_case(11, n)
    dz = O.softmax_logits_bwd(z, dy)
    fd = _fd_grad(O.softmax, z, dy)
    assert np.abs(dz - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max())
    assert np.array_equal(dz, O.softmax_bwd(O.softmax(z), dy))  # the composition it is defined as


@pytest.mark.parametrize("n", [2, 7, 33])
def test_xent_bwd_matches_finite_differences(n):
    r = _rng(12)
    z = r.standard_normal((3, n)) * 3.0
    t = r.uniform(0.0, 1.0, (3, n))            # soft labels that do not sum to one
    w = np.array([1.0, 0.5, -2.0])
    dz = O.xent_bwd(z, t, w)
    h = 1e-5
    fd = np.empty_like(z)
    for k in range(n):
        zp, zm = z.copy(), z.copy()
        zp[:, k] += h
        zm[:, k] -= h
        fd[:, k] = w * (_xent_loss(zp, t) - _xent_loss(zm, t)) / (2 * h)
    assert np.abs(dz - fd).max() <= 1e-8 * max(1.0, np.abs(fd).max())


def test_logits_gradients_against_torch_and_special_cases():
    r = _rng(13)
    z = r.standard_normal((4, 200)) * 3.0
    dy = r.standard_normal((4, 200))
    t = r.dirichlet(np.ones(200), size=4)        # probability targets
    w = r.uniform(0.5, 2.0, 4)
    tz = torch.tensor(z, requires_grad=True)
    torch.softmax(tz, dim=1).backward(torch.tensor(dy))
    assert np.allclose(O.softmax_logits_bwd(z, dy), tz.grad.numpy(), rtol=1e-12, atol=1e-15)
    tz = torch.tensor(z, requires_grad=True)
    F.cross_entropy(tz, torch.tensor(t), reduction="none").backward(torch.tensor(w))
    assert np.allclose(O.xent_bwd(z, t, w), tz.grad.numpy(), rtol=1e-12, atol=1e-15)
    # shift invariance: the gradients sum to zero
    assert np.abs(O.softmax_logits_bwd(z, dy).sum(axis=1)).max() <= 1e-14
    assert np.abs(O.xent_bwd(z, t, w).sum(axis=1)).max() <= 1e-14
    # the target equal to the prediction: no gradient; a one-hot target: y - e_k
    assert np.abs(O.xent_bwd(z, O.softmax(z))).max() <= 1e-16
    onehot = np.zeros_like(z)
    onehot[np.arange(4), [3, 50, 100, 199]] = 1.0
    assert np.allclose(O.xent_bwd(z, onehot), O.softmax(z) - onehot, rtol=0, atol=1e-16)


@pytest.mark.parametrize("dtype", [O.F32, O.BF16])
def test_batch_driver_logits_ops(dtype):
    r = _rng(14)
    rows, cols = 5, 61
    z = (r.standard_normal((rows, cols)) * 3).astype(np.float32)
    d = r.uniform(0, 1, (rows, cols)).astype(np.float32)
    w = r.uniform(0.5, 2, rows).astype(np.float32)
    if dtype == O.BF16:
        zr = torch.from_numpy(z).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        dr = torch.from_numpy(d).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
        zd, dd = O.bf16_to_double(zr), O.bf16_to_double(dr)
    else:
        zr, dr, zd, dd = z, d, z.astype(np.float64), d.astype(np.float64)
    dx64, _ = O.run_bwd(O.SOFTMAX_LOGITS, dtype, zr, dr, rows, cols)
    assert np.array_equal(dx64, O.softmax_logits_bwd(zd, dd))
    dx64, _ = O.run_bwd(O.XENT, dtype, zr, dr, rows, cols, rstd=w)
    assert np.array_equal(dx64, O.xent_bwd(zd, dd, w.astype(np.float64)))
    dx64, _ = O.run_bwd(O.XENT, dtype, zr, dr, rows, cols)  # no scale: 1
    assert np.array_equal(dx64, O.xent_bwd(zd, dd))
