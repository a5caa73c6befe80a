"""Pins of the FP64 MLP oracle: a hand-built network with a known output,
central finite differences of the loss (an independent check of backprop),
and Adam's closed-form first step."""
import numpy as np
import pytest

import oracle.mlp as M


def test_hand_built_network():
    n_in = 3
    p = np.zeros(M.n_params(n_in))
    layers = M.unflatten(p, n_in)  # views into p
    layers[0][0][0, 0] = 1.0       # h1[0] = relu(x0)
    layers[1][0][0, 0] = 1.0       # h2[0] = relu(h1[0])
    layers[2][0][0, 0] = 1.0       # h3[0] = relu(h2[0])
    layers[3][0][0, 0] = 2.0       # y = 2 h3[0] + 1
    layers[3][1][0] = 1.0
    y, _ = M.forward(p, np.array([[3.0, 5.0, -1.0], [-3.0, 9.0, 9.0], [0.5, 0.0, 0.0]]))
    assert np.allclose(y, [7.0, 1.0, 2.0], rtol=0, atol=1e-15)
    assert M.n_params(18) == 18 * 64 + 64 + 2 * (64 * 64 + 64) + 64 + 1


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, n = 5, 7
    p = rng.standard_normal(M.n_params(n_in)) * 0.3
    X = rng.standard_normal((n, n_in))
    t = rng.standard_normal(n)
    loss, g = M.loss_and_grad(p, X, t)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (M.loss_and_grad(p + e, X, t)[0] - M.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    assert loss == pytest.approx(np.mean((M.forward(p, X)[0] - t) ** 2))


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3])
    p1, m, v = M.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), t=1, lr=0.1, eps=0.0)
    # bias-corrected m = g, v = g^2, so the first step is -lr * sign(g)
    assert np.allclose(p1, -0.1 * np.sign(g), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
