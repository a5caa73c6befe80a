"""FP64 reference of the latency MLP (forward, backward, MSE, Adam).

TEST INFRASTRUCTURE ONLY: the product trains and evaluates the network with
its own CUDA kernels (`credit_mlp_*`); this numpy restatement checks them.

Network: n_in -> 64 -> 64 -> 64 -> 1, ReLU on the hidden layers, linear
output.  Flat parameter layout, layer by layer: W (out x in, row-major), then
b (out).  Loss: mean squared error L = (1/n) sum_i (y_i - t_i)^2.
Adam (Kingma & Ba, 2015): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
DEPTH = 3


def layer_dims(n_in: int, hidden: int = HIDDEN, depth: int = DEPTH):
    dims = [n_in] + [hidden] * depth + [1]
    return list(zip(dims[:-1], dims[1:]))


def n_params(n_in: int, hidden: int = HIDDEN, depth: int = DEPTH) -> int:
    return sum(o * i + o for i, o in layer_dims(n_in, hidden, depth))


def unflatten(params: np.ndarray, n_in: int, hidden: int = HIDDEN, depth: int = DEPTH):
    out, k = [], 0
    for i, o in layer_dims(n_in, hidden, depth):
        W = params[k:k + o * i].reshape(o, i)
        k += o * i
        b = params[k:k + o]
        k += o
        out.append((W, b))
    return out


def forward(params, X, hidden=HIDDEN, depth=DEPTH):
    """Returns (y (n,), activations list [input, h1, h2, h3])."""
    X = np.asarray(X, dtype=np.float64)
    layers = unflatten(np.asarray(params, dtype=np.float64), X.shape[1], hidden, depth)
    acts = [X]
    a = X
    for li, (W, b) in enumerate(layers):
        z = a @ W.T + b
        if li < len(layers) - 1:
            a = np.maximum(z, 0.0)
            acts.append(a)
        else:
            a = z
    return a[:, 0], acts


def loss_and_grad(params, X, t, hidden=HIDDEN, depth=DEPTH):
    """MSE loss and its gradient with respect to the flat parameters."""
    params = np.asarray(params, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = X.shape[0]
    y, acts = forward(params, X, hidden, depth)
    loss = float(np.mean((y - t) ** 2))
    layers = unflatten(params, X.shape[1], hidden, depth)
    delta = (2.0 / n) * (y - t)[:, None]          # dL/dz of the output layer
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        a_in = acts[li]
        gW = delta.T @ a_in
        gb = delta.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            delta = (delta @ W) * (acts[li] > 0.0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def adam_step(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
