"""The allocation-free two-pass entry point against the regular one.

credit_run_two_pass_noalloc serves callers that cannot allocate device
memory (a framework's caching allocator owns the device heap, or an
embedding forbids allocation after start-up).  It must give the same results as the
split-row two-pass plan of credit_run_ex, call after call, even though every
call reuses one fixed scratch array.  This file is collected last so that a
failure here cannot hide the other tests' results.
"""
import pytest
import torch

from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2609_01864_gb300 import build as B
    B.build()
    yield


CASES = [(C.SOFTMAX, C.F32, 300, 20000, 3), (C.LOGSUMEXP, C.BF16, 257, 12345, 4),
         (C.LAYERNORM, C.F32, 129, 40000, 5), (C.RMSNORM, C.BF16, 70000, 512, 4)]


@pytest.mark.parametrize("op,dt,rows,cols,G", CASES)
def test_noalloc_matches_the_workspace_path_twice(op, dt, rows, cols, G):
    x, s = U.make_input(dt, rows, cols, kind="outliers" if op in (C.LAYERNORM, C.RMSNORM) else "normal",
                        std=2.0, seed=cols)
    xd = x.cuda()
    g, b = synth.gamma_beta(cols, seed=3)
    kw = dict(gamma=g.cuda() if op in (C.LAYERNORM, C.RMSNORM) else None,
              beta=b.cuda() if op == C.LAYERNORM else None)
    shape = (rows,) if op == C.LOGSUMEXP else (rows, cols)
    odt = torch.float32 if op == C.LOGSUMEXP else xd.dtype
    ref = torch.empty(shape, device="cuda", dtype=odt)
    C.run_ex(op, xd, ref, plan=C.make_plan(C.PATH_TWO_PASS, ctas_per_row=G), **kw)
    y64_ref = U.reference(op, C.DTYPE_OF[x.dtype], x, s, g if kw["gamma"] is not None else None,
                          b if kw["beta"] is not None else None)
    out_dtype = C.F32 if op == C.LOGSUMEXP else C.DTYPE_OF[x.dtype]
    for _ in range(2):  # two calls in a row share (and overwrite) the scratch
        out = torch.full(shape, float("nan"), device="cuda", dtype=odt)
        assert C.run_two_pass_noalloc(op, xd, out, G, **kw) == C.OK
        torch.cuda.synchronize()
        # same kernels, same partial order: identical to the workspace path
        assert torch.equal(out, ref)
        assert U.error_metric(op, out_dtype, U.to64(out), y64_ref, x64=U.decoded(x, s) if op == C.LAYERNORM else None,
                              gamma=g, beta=b) <= 1.0


@pytest.mark.parametrize("op", [C.LAYERNORM, C.RMSNORM], ids=["layernorm", "rmsnorm"])
def test_noalloc_fp8_output_matches_the_workspace_path_twice(op):
    """FP8-E4M3 output of the norms: the amax stage between the two sweeps and the per-row output scale,
    written at each launch's row offset (70000 rows at G = 4 take two launches)."""
    rows, cols, G = 70000, 600, 4
    x, _ = U.make_input(C.BF16, rows, cols, kind="outliers", seed=11)
    xd = x.cuda()
    g, b = synth.gamma_beta(cols, seed=3)
    kw = dict(gamma=g.cuda(), beta=b.cuda() if op == C.LAYERNORM else None, out_dtype=C.FP8_E4M3)
    ref = torch.empty(rows, cols, device="cuda", dtype=torch.float8_e4m3fn)
    ref_s = torch.empty(rows, device="cuda")
    C.run_ex(op, xd, ref, plan=C.make_plan(C.PATH_TWO_PASS, ctas_per_row=G), out_scale=ref_s, **kw)
    pick = torch.arange(0, rows, 997)
    y64_ref = U.reference(op, C.BF16, x[pick], None, g, b if op == C.LAYERNORM else None)
    for _ in range(2):
        out = torch.zeros(rows, cols, device="cuda", dtype=torch.float8_e4m3fn)
        osc = torch.full((rows,), float("nan"), device="cuda")
        assert C.run_two_pass_noalloc(op, xd, out, G, out_scale=osc, **kw) == C.OK
        torch.cuda.synchronize()
        assert torch.equal(out.view(torch.uint8), ref.view(torch.uint8)) and torch.equal(osc, ref_s)
        assert U.error_metric(op, C.FP8_E4M3, U.to64(out[pick]), y64_ref, osc[pick].cpu().numpy()) <= 1.0


def test_noalloc_rejects_out_of_range_split_and_bad_args():
    x = torch.randn(4, 1024, device="cuda")
    y = torch.empty_like(x)
    assert C.run_two_pass_noalloc(C.SOFTMAX, x, y, 1) == C.ERR_UNSUPPORTED
    assert C.run_two_pass_noalloc(C.SOFTMAX, x, y, 4097) == C.ERR_UNSUPPORTED
    assert C.run_two_pass_noalloc(C.SOFTMAX, x, y, 4, rows=4, cols=0) == C.ERR_INVALID_ARG
