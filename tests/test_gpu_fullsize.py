"""Parity at the full workload sizes, on sampled rows.

Inputs are generated on the device (seeded) at the sizes of the benchmark
workload (4096 rows x {16K .. 512K} FP32 LayerNorm / RMSNorm with gamma/beta
and 1% outliers) and of the precision workload (4096 rows x {128K, 256K}
softmax / log-sum-exp over BF16 and per-row-scaled FP8-E4M3 logits ~ N(0, 3^2)).
Each case runs once through the C ABI with the plan the planner picks (the
launch configuration bench.py times) and once on the cluster path; 12 seeded
rows are checked element by element against the FP64 oracle, and the row-wise
invariants (softmax sums to 1) are checked on every row.
"""
import os

import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

import parity_util as U

pytestmark = pytest.mark.gpu
ROWS = 4096


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    C.load_model(os.path.join(os.path.dirname(C.__file__), "data", "gb300.calib"))
    yield
    torch.cuda.empty_cache()


def sample_rows(n=12, seed=0):
    rng = np.random.default_rng(seed)
    return sorted(set(rng.choice(ROWS, n - 2, replace=False).tolist() + [0, ROWS - 1]))


def cluster_plan(op, x, y, kw):
    for P in (2, 4, 8, 16):
        p = C.make_plan(C.PATH_CLUSTER, P)
        if C.plan_check(op, x, y, p, **kw) == C.OK:
            return p
    return None


@pytest.mark.parametrize("cols", [16384, 65536, 131072, 262144, 524288])
@pytest.mark.parametrize("op", [C.LAYERNORM, C.RMSNORM])
def test_config2_sampled_rows(op, cols):
    x = synth.outliers(ROWS, cols, seed=synth.SEED_DATA, device="cuda")
    g, b = synth.gamma_beta(cols, device="cuda")
    kw = dict(gamma=g, beta=b if op == C.LAYERNORM else None)
    y = torch.empty_like(x)
    pick = sample_rows(seed=cols)
    xs = x[pick].cpu()
    ref = U.reference(op, C.F32, xs, None, g.cpu(), b.cpu() if op == C.LAYERNORM else None)
    plans = [None]
    cp = cluster_plan(op, x, y, kw)
    if cp is not None:
        plans.append(cp)
    for plan in plans:
        y.fill_(float("nan"))
        C.run_ex(op, x, y, plan=plan, **kw)
        torch.cuda.synchronize()
        assert C.device_error() == C.OK
        assert U.error_metric(op, C.F32, U.to64(y[pick]), ref) <= 1.0
        assert not torch.isnan(y).any()
    del x, y


@pytest.mark.parametrize("cols", [131072, 262144])
@pytest.mark.parametrize("dt", [C.BF16, C.FP8_E4M3])
@pytest.mark.parametrize("op", [C.SOFTMAX, C.LOGSUMEXP])
def test_config3_sampled_rows(op, dt, cols):
    x32 = synth.normal(ROWS, cols, std=3.0, seed=synth.SEED_DATA, device="cuda")
    if dt == C.BF16:
        x, sc = synth.to_bf16(x32), None
    else:
        x, sc = synth.to_e4m3_rowscaled(x32)
    del x32
    out_dt = C.F32 if op == C.LOGSUMEXP else dt
    pick = sample_rows(seed=cols + dt)
    xs = x[pick].cpu()
    ss = None if sc is None else sc[pick].cpu()
    ref = U.reference(op, dt, xs, ss)
    shape = (ROWS,) if op == C.LOGSUMEXP else (ROWS, cols)
    y = torch.empty(shape, device="cuda", dtype=C.TORCH_DTYPE[out_dt])
    osc = torch.empty(ROWS, device="cuda") if out_dt == C.FP8_E4M3 else None
    kw = dict(in_dtype=dt, out_dtype=out_dt, in_scale=sc, out_scale=osc)
    plans = [None]
    cp = cluster_plan(op, x, y, kw)
    if cp is not None:
        plans.append(cp)
    for plan in plans:
        C.run_ex(op, x, y, plan=plan, **kw)
        torch.cuda.synchronize()
        assert C.device_error() == C.OK
        ys = U.to64(y[pick])
        m = U.error_metric(op, out_dt, ys, ref, None if osc is None else osc[pick].cpu().numpy())
        assert m <= 1.0, (plan, m)
        if op == C.SOFTMAX:
            sums = y.float().sum(dim=1) if osc is None else (y.float() * osc[:, None]).sum(dim=1)
            tol = 5e-2 if osc is not None else 1e-2  # sum of rounded BF16 / E4M3 outputs
            assert torch.max(torch.abs(sums - 1)).item() <= tol
    del x, y
