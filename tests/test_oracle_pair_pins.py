"""Pins of the oracle's two-input statistics and their gradients: the
weighted variance and the Pearson correlation of a row pair (the
"weighted-variance backward" and "Pearson-correlation backward" workloads).

The forward values are pinned to numpy's own routines (np.cov with analytic
weights and bias=True, np.corrcoef); the gradients to central differences of
those forwards, to torch float64 autograd, to the invariances that fix
directions the gradient must be orthogonal to (shift of x; positive scale of
x or y for the correlation; scale of the weights for the weighted variance),
and to closed forms on tiny rows.
"""
import numpy as np
import pytest
import torch

import oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


def test_forwards_match_numpy():
    r = _rng(1)
    x = r.standard_normal((4, 37)) * 3 + 10
    y = 0.5 * x + r.standard_normal((4, 37))
    w = r.uniform(0.1, 2.0, (4, 37))
    assert np.allclose(O.wvar(x, w), [np.cov(x[i], aweights=w[i], bias=True) for i in range(4)], rtol=1e-13)
    assert np.allclose(O.pearson(x, y), [np.corrcoef(x[i], y[i])[0, 1] for i in range(4)], rtol=1e-13)


def _fd(f, a, h=1e-6):
    g = np.empty_like(a)
    for k in range(a.shape[1]):
        ap, am = a.copy(), a.copy()
        ap[:, k] += h
        am[:, k] -= h
        g[:, k] = (f(ap) - f(am)) / (2 * h)
    return g


@pytest.mark.parametrize("n", [2, 9, 40])
def test_wvar_gradients_match_finite_differences(n):
    r = _rng(2)
    x = r.standard_normal((3, n)) * 2
    w = r.uniform(0.1, 2.0, (3, n))
    g = np.array([1.0, -0.5, 2.0])
    dx, dw = O.wvar_bwd(x, w, g)
    fdx = g[:, None] * _fd(lambda v: O.wvar(v, w), x)
    fdw = g[:, None] * _fd(lambda v: O.wvar(x, v), w)
    assert np.abs(dx - fdx).max() <= 1e-7 * max(1.0, np.abs(fdx).max())
    assert np.abs(dw - fdw).max() <= 1e-7 * max(1.0, np.abs(fdw).max())


@pytest.mark.parametrize("n", [3, 9, 40])
def test_pearson_gradients_match_finite_differences(n):
    r = _rng(3)
    x = r.standard_normal((3, n))
    y = 0.3 * x + r.standard_normal((3, n))
    g = np.array([1.0, 0.25, -3.0])
    dx, dy = O.pearson_bwd(x, y, g)
    fdx = g[:, None] * _fd(lambda v: O.pearson(v, y), x)
    fdy = g[:, None] * _fd(lambda v: O.pearson(x, v), y)
    assert np.abs(dx - fdx).max() <= 1e-7 * max(1.0, np.abs(fdx).max())
    assert np.abs(dy - fdy).max() <= 1e-7 * max(1.0, np.abs(fdy).max())


def test_torch_float64_autograd_agrees():
    r = _rng(4)
    x = r.standard_normal((3, 64))
    y = 0.5 * x + r.standard_normal((3, 64))
    w = r.uniform(0.1, 2.0, (3, 64))
    tx, tw = torch.tensor(x, requires_grad=True), torch.tensor(w, requires_grad=True)
    mu = (tw * tx).sum(1, keepdim=True) / tw.sum(1, keepdim=True)
    v = (tw * (tx - mu) ** 2).sum(1) / tw.sum(1)
    v.sum().backward()
    dx, dw = O.wvar_bwd(x, w)
    assert np.allclose(dx, tx.grad.numpy(), rtol=1e-12, atol=1e-14)
    assert np.allclose(dw, tw.grad.numpy(), rtol=1e-12, atol=1e-14)
    tx, ty = torch.tensor(x, requires_grad=True), torch.tensor(y, requires_grad=True)
    rr = torch.stack([torch.corrcoef(torch.stack([tx[i], ty[i]]))[0, 1] for i in range(3)])
    rr.sum().backward()
    dx, dy = O.pearson_bwd(x, y)
    assert np.allclose(dx, tx.grad.numpy(), rtol=1e-11, atol=1e-13)
    assert np.allclose(dy, ty.grad.numpy(), rtol=1e-11, atol=1e-13)


def test_gradients_are_orthogonal_to_the_invariant_directions():
    r = _rng(5)
    x = r.standard_normal((4, 50)) * 2 + 3
    y = -0.4 * x + r.standard_normal((4, 50))
    w = r.uniform(0.1, 2.0, (4, 50))
    dx, dw = O.wvar_bwd(x, w)
    assert np.abs(dx.sum(1)).max() <= 1e-14            # v(x + c) = v(x)
    assert np.abs((dw * w).sum(1)).max() <= 1e-14      # v(x; c w) = v(x; w)
    dx, dy = O.pearson_bwd(x, y)
    xc, yc = x - x.mean(1, keepdims=True), y - y.mean(1, keepdims=True)
    assert np.abs(dx.sum(1)).max() <= 1e-14 and np.abs(dy.sum(1)).max() <= 1e-14   # shifts
    assert np.abs((dx * xc).sum(1)).max() <= 1e-14 and np.abs((dy * yc).sum(1)).max() <= 1e-14  # scales


def test_closed_forms():
    # two points: the correlation is +-1 and its gradient vanishes
    x, y = np.array([[0.0, 1.0]]), np.array([[2.0, 5.0]])
    assert O.pearson(x, y)[0] == pytest.approx(1.0, abs=1e-15)
    dx, dy = O.pearson_bwd(x, y)
    assert np.abs(dx).max() <= 1e-15 and np.abs(dy).max() <= 1e-15
    # unit weights: the population variance, dx = 2 (x - mean) / N
    x = np.array([[1.0, 2.0, 4.0, 9.0]])
    w = np.ones_like(x)
    assert O.wvar(x, w)[0] == pytest.approx(np.var(x), rel=1e-15)
    dx, dw = O.wvar_bwd(x, w)
    assert np.allclose(dx, 2 * (x - x.mean()) / 4, rtol=1e-15)
    assert np.allclose(dw, ((x - x.mean()) ** 2 - np.var(x)) / 4, rtol=1e-14)
