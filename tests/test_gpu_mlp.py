"""GPU MLP kernels against the FP64 oracle (oracle/mlp.py): the loss and its
gradient from one forward + backward, training progress, and save / load."""
import numpy as np
import pytest

import oracle.mlp as OM
from paper_2609_01864_gb300 import credit as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield


def test_gradient_matches_fp64_backprop():
    rng = np.random.default_rng(1)
    n_in = C.MLP_FEATURES
    assert C.mlp_num_params() == OM.n_params(n_in)
    p = (rng.standard_normal(OM.n_params(n_in)) * 0.2).astype(np.float32)
    X = rng.standard_normal((37, n_in)).astype(np.float32)
    t = rng.standard_normal(37).astype(np.float32)
    loss, g = C.mlp_grad(p, X, t)
    ref_loss, ref_g = OM.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    scale = np.max(np.abs(ref_g))
    assert np.max(np.abs(g - ref_g)) <= 1e-3 * scale


def test_training_reduces_loss_and_predicts():
    rng = np.random.default_rng(2)
    n = 4096
    X = rng.standard_normal((n, C.MLP_FEATURES)).astype(np.float32)
    y = (np.maximum(X[:, 0], 0) * 2 + X[:, 1] - 0.5 * X[:, 2]).astype(np.float32)
    curve = C.mlp_train(X, y, epochs=60, batch=256, lr=3e-3, seed=0)
    assert curve[-1] < 0.1 * curve[0]
    pred = C.mlp_predict(X[:256])
    assert np.mean((pred - y[:256]) ** 2) < 0.05 * np.var(y)


def test_save_and_load_roundtrip(tmp_path):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((512, C.MLP_FEATURES)).astype(np.float32)
    y = X[:, 0].astype(np.float32)
    C.mlp_train(X, y, epochs=5, batch=128, seed=1)
    a = C.mlp_predict(X[:64])
    path = str(tmp_path / "m.mlp")
    C.mlp_save(path)
    C.mlp_train(X, -y, epochs=5, batch=128, seed=2)   # different weights
    C.mlp_load(path)
    b = C.mlp_predict(X[:64])
    assert np.allclose(a, b, rtol=1e-5, atol=1e-5)


def test_ensemble_is_the_mean_of_its_members(tmp_path):
    rng = np.random.default_rng(4)
    X = rng.standard_normal((1024, C.MLP_FEATURES)).astype(np.float32)
    y = (X[:, 0] - 2 * X[:, 3]).astype(np.float32)
    members = []
    for seed in (7, 8, 9):
        C.mlp_train(X, y, epochs=8, batch=128, seed=seed)
        members.append(C.mlp_predict(X[:64]))
    C.mlp_train_ensemble(X, y, members=3, epochs=8, batch=128, seed=7)
    assert C.mlp_members() == 3
    ens = C.mlp_predict(X[:64])
    assert np.allclose(ens, np.mean(members, axis=0), rtol=1e-4, atol=1e-4)
    path = str(tmp_path / "e.mlp")
    C.mlp_save(path)
    C.mlp_train(X, -y, epochs=2, batch=128, seed=1)  # one different network
    assert C.mlp_members() == 1
    C.mlp_load(path)
    assert C.mlp_members() == 3
    assert np.allclose(C.mlp_predict(X[:64]), ens, rtol=1e-5, atol=1e-5)
