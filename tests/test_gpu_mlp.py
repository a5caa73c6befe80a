"""GPU MLP kernels against the FP64 oracle (oracle/mlp.py): the loss and its
gradient from one forward + backward, training progress, and save / load."""
import os

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


DATA = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2609_01864_gb300", "data")


def read_weights(path):
    """The ensemble file as written by credit_mlp_save (version 2): per member the feature mean / std pairs,
    the target mean / std, then the flat parameters."""
    with open(path) as f:
        head = f.readline().split()
        assert head[0] == "credit-mlp" and head[1] == "2"
        n_in, n_par, members = int(head[2]), int(head[4]), int(head[5])
        vals = np.array(f.read().split(), dtype=np.float64)
    out, k = [], 0
    for _ in range(members):
        fm = vals[k:k + 2 * n_in:2]
        fs = vals[k + 1:k + 2 * n_in:2]
        k += 2 * n_in
        tm, ts = vals[k], vals[k + 1]
        k += 2
        out.append((fm, fs, tm, ts, vals[k:k + n_par]))
        k += n_par
    assert k == len(vals)
    return out


def test_predict_matches_fp64_forward_per_sample():
    """credit_mlp_predict of the committed ensemble, sample by sample, against the FP64 forward of the same
    weights (features of 300 sweep candidates): error <= 1e-5 of max(|y*|, 1) in log2 latency (the outputs are
    latencies relative to a shape's mean, near 0, as LSE outputs can be: the FP32 bound of reading r7)."""
    from paper_2609_01864_gb300 import sweep as S
    path = os.path.join(DATA, "gb300_mlp.txt")
    C.mlp_load(path)
    rows = S.read_csv(os.path.join(DATA, "sweep_gb300.csv"))
    pick = np.random.default_rng(5).choice(len(rows), 300, replace=False)
    X = np.stack([S.features_of(rows[i]) for i in pick]).astype(np.float32)
    got = C.mlp_predict(X).astype(np.float64)
    ref = np.zeros(len(X))
    members = read_weights(path)
    for fm, fs, tm, ts, p in members:
        xs = (X.astype(np.float64) - fm) / fs
        ref += OM.forward(p, xs)[0] * ts + tm
    ref /= len(members)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) <= 1e-5


@pytest.mark.parametrize("step", [1, 7, 1000])
def test_adam_step_matches_fp64(step):
    """One step of the training kernel's Adam update against oracle.mlp.adam_step, each result within a few
    FP32 roundings of the magnitudes of its terms: m = b1 m + (1 - b1) g and v = b2 v + (1 - b2) g^2 to
    4 * 2^-24 of (b1 |m| + (1 - b1) |g|) and of (b2 v + (1 - b2) g^2); the parameters to 2^-23 of |p| plus
    16 * 2^-24 of the step lr mh / (sqrt(vh) + eps) plus the first moment's rounding carried through it."""
    rng = np.random.default_rng(step)
    n = C.mlp_num_params()
    p = rng.standard_normal(n).astype(np.float32)
    g = (rng.standard_normal(n) * np.exp(rng.uniform(-8, 2, n))).astype(np.float32)
    m = (rng.standard_normal(n) * 0.1).astype(np.float32)
    v = (np.abs(rng.standard_normal(n)) * 0.01).astype(np.float32)
    lr = 2e-3
    p2, m2, v2 = C.mlp_adam_step(p, g, m, v, step, lr)
    # the kernel's hyperparameters are the FP32 values of 0.9, 0.999, 1e-8 and lr (1 - b1 is then
    # 0.10000002, not 0.1): the oracle takes the same values
    f32 = lambda z: float(np.float32(z))  # noqa: E731
    rp, rm, rv = OM.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                              v.astype(np.float64), step, lr=f32(lr), b1=f32(0.9), b2=f32(0.999), eps=f32(1e-8))
    u = 2.0 ** -24
    m64, v64, g64 = m.astype(np.float64), v.astype(np.float64), g.astype(np.float64)
    assert np.all(np.abs(m2 - rm) <= 4 * u * (0.9 * np.abs(m64) + 0.1 * np.abs(g64)))
    assert np.all(np.abs(v2 - rv) <= 4 * u * (0.999 * v64 + 0.001 * g64 * g64))
    step_ref = np.abs(rp - p.astype(np.float64))
    # the moment's own rounding (above), carried through the step: lr dm / c1 / (sqrt(vh) + eps)
    c1, c2 = 1 - f32(0.9) ** step, 1 - f32(0.999) ** step
    dm = 4 * u * (0.9 * np.abs(m64) + 0.1 * np.abs(g64))
    carried = lr * dm / c1 / (np.sqrt(rv / c2) + 1e-8)
    assert np.all(np.abs(p2 - rp) <= 2 * u * np.abs(rp) + 16 * u * step_ref + carried)
    assert np.max(np.abs(p2 - p)) > 0.1 * lr  # the step moved the parameters


def test_learned_model_beats_the_analytic_model_on_held_out_shapes():
    """On the committed sweep's held-out 20% of shapes (seeded split by shape), the committed learned model's
    picks are within 5% of the measured best more often than the analytic model's (Eq. 7-9), and reach the
    accuracy recorded in the committed summary."""
    import json
    from paper_2609_01864_gb300 import sweep as S
    from paper_2609_01864_gb300 import synth
    C.load_model(os.path.join(DATA, "gb300.calib"))
    rows = S.read_csv(os.path.join(DATA, "sweep_gb300.csv"))
    summary = json.load(open(os.path.join(DATA, "sweep_gb300_summary.json")))
    # the split covers the log-uniform shapes only; shape ids from summary["shapes"] on are training-only
    _, test = synth.split_by_shape(summary["shapes"])
    acc, n = S.evaluate(rows, test)
    assert n == summary["test_shapes"]
    assert acc["learned"] > acc["analytic"] > 0.0
    assert acc["learned"] == pytest.approx(summary["pick_accuracy"]["learned"], abs=1e-9)


def test_plan_cache_repeats_the_choice_and_follows_model_changes(monkeypatch):
    """A call without a plan reuses the plan chosen for the same shape; loading a calibration or training a
    model empties the cache, and CREDIT_MODEL bypasses it."""
    import time
    calib = os.path.join(DATA, "gb300.calib")
    C.load_model(calib)
    shape = (C.LAYERNORM, 4096, 65536, C.F32)
    p1 = C.plan(*shape)
    t0 = time.perf_counter()
    for _ in range(200):
        p = C.plan(*shape)
    dt = (time.perf_counter() - t0) / 200
    assert p.as_dict() == p1.as_dict()
    assert dt < 50e-6, f"cached plan took {dt * 1e6:.1f} us"
    monkeypatch.setenv("CREDIT_MODEL", "analytic")
    pa = C.plan(*shape)
    assert pa.source != 1  # the analytic model's plan, not the cached learned one
    monkeypatch.delenv("CREDIT_MODEL")
    assert C.plan(*shape).as_dict() == p1.as_dict()
    # a different (tiny, random) model: the next plan is the new model's
    rng = np.random.default_rng(5)
    X = rng.standard_normal((512, C.MLP_FEATURES)).astype(np.float32)
    C.mlp_train_ensemble(X, rng.standard_normal(512).astype(np.float32), members=1, epochs=2)
    p2 = C.plan(*shape)
    assert p2.source == 1 and p2.as_dict() != p1.as_dict()
    C.load_model(calib)  # back to the committed model: the first choice again
    assert C.plan(*shape).as_dict() == p1.as_dict()
