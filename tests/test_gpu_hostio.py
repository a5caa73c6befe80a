"""GPU tests of credit_run_host: the ops on host buffers, streamed through the
library's device staging slots in blocks (copy-in, op and copy-out of
consecutive blocks overlapped on three streams).

Results are checked against the FP64 oracle and, for rows whose byte
length is a multiple of 16, bit for bit against credit_run_ex with the same
plan on device copies of the same data (same kernels; rows are independent;
a ragged row is sliced on the 16-byte grid of its own address, which the
staging buffers do not preserve, so its reduction order may differ).
Shapes give several blocks and more blocks than staging slots (slot reuse),
strided rows, FP8 scales in and out, and pageable as well as pinned memory.
"""
import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def host(t, pinned=True):
    h = torch.empty(t.shape, dtype=t.dtype, pin_memory=pinned)
    h.copy_(t)
    return h


def affine(op, cols, pinned=True):
    if op in (C.LAYERNORM, C.RMSNORM):
        g, b = synth.gamma_beta(cols, seed=4)
        return host(g, pinned), (host(b, pinned) if op == C.LAYERNORM else None)
    return None, None


PLANS = {"auto": None, "two_pass_g2": C.make_plan(C.PATH_TWO_PASS, ctas_per_row=2),
         "cluster4": C.make_plan(C.PATH_CLUSTER, 4)}


@pytest.mark.parametrize("cols", [4099, 4112])
@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("op", [C.SOFTMAX, C.LOGSUMEXP, C.LAYERNORM, C.RMSNORM])
@pytest.mark.parametrize("dt", [(C.F32, C.F32), (C.BF16, C.BF16), (C.FP8_E4M3, C.F32), (C.F32, C.FP8_E4M3)],
                         ids=lambda d: f"{d[0]}to{d[1]}")
def test_host_buffers_match_oracle_and_device_path(op, dt, plan, cols):
    tin, tout = dt
    if op == C.LOGSUMEXP:
        tout = C.F32
    rows = 37  # 8 blocks of 5 rows through 3 slots
    x, s = U.make_input(tin, rows, cols, kind="outliers" if op in (C.LAYERNORM, C.RMSNORM) else "normal", std=3.0,
                        seed=rows + cols + tin * 7 + tout)
    g, b = affine(op, cols)
    hx = host(x)
    hs = None if s is None else host(s)
    shape = (rows,) if op == C.LOGSUMEXP else (rows, cols)
    hy = torch.empty(shape, dtype=C.TORCH_DTYPE[tout], pin_memory=True)
    hos = torch.empty(rows, pin_memory=True) if (tout == C.FP8_E4M3 and op != C.LOGSUMEXP) else None
    C.run_host(op, hx, hy, plan=PLANS[plan], in_dtype=tin, out_dtype=tout, in_scale=hs, out_scale=hos, gamma=g,
               beta=b)
    ref = U.reference(op, tin, x, s, g, b)
    assert U.error_metric(op, tout, U.to64(hy), ref, None if hos is None else hos.numpy(),
                          x64=U.decoded(x, s) if op == C.LAYERNORM else None,
                          gamma=None if g is None else g.cpu(), beta=None if b is None else b.cpu()) <= 1.0
    # the same plan on device buffers gives the same bits
    p = PLANS[plan] if PLANS[plan] is not None else C.plan(op, -(-rows // 8), cols, tin, tout)
    dy, dos = U.run_gpu(op, x, s, out_dtype=tout, plan=p, gamma=g, beta=b)
    torch.cuda.synchronize()
    isz = {C.F32: 4, C.BF16: 2, C.FP8_E4M3: 1}[tin]
    if dy is not None and (cols * isz) % 16 == 0:
        assert torch.equal(dy.cpu().view(torch.uint8), hy.view(torch.uint8))
        if hos is not None:
            assert torch.equal(dos.cpu(), hos)


def test_strided_rows_pageable_memory_and_slot_reuse():
    rows, cols, ld = 301, 5003, 5011
    op = C.RMSNORM
    base = synth.normal(rows, ld, seed=9)
    hx = base.contiguous()  # pageable
    hy = torch.full((rows, ld), float("nan"))
    g, _ = affine(op, cols, pinned=False)
    C.run_host(op, hx, hy, rows=rows, cols=cols, ld_in=ld, ld_out=ld, in_dtype=C.F32, out_dtype=C.F32, gamma=g)
    ref = U.reference(op, C.F32, hx[:, :cols].contiguous(), None, g, None)
    assert U.error_metric(op, C.F32, hy[:, :cols].double().numpy(), ref) <= 1.0
    assert torch.isnan(hy[:, cols:]).all()  # the padding between rows is not written


def test_many_blocks_of_a_wide_shape_sampled():
    rows, cols = 1500, 131072  # 188-row blocks, 8 of them
    op = C.LAYERNORM
    x = synth.outliers(rows, cols, seed=3)
    hx = host(x)
    hy = torch.empty(rows, cols, pin_memory=True)
    g, b = affine(op, cols)
    C.run_host(op, hx, hy, gamma=g, beta=b)
    pick = [0, 1, 187, 188, 700, 1499]
    ref = U.reference(op, C.F32, x[pick], None, g, b)
    assert U.error_metric(op, C.F32, U.to64(hy[pick]), ref) <= 1.0


def test_zero_rows_and_bad_arguments():
    hx = torch.zeros(0, 64)
    assert C.run_host(C.SOFTMAX, hx, hx, rows=0, cols=64) == C.OK
    hx = torch.zeros(4, 64, pin_memory=True)
    hl = torch.zeros(4, pin_memory=True)
    with pytest.raises(C.CreditError):
        C.run_host(C.LOGSUMEXP, hx, hx, rows=4, cols=64)  # logsumexp in place
    with pytest.raises(C.CreditError):
        C.run_host(C.SOFTMAX, hx, hl, rows=4, cols=64, plan=C.make_plan(C.PATH_CLUSTER, 17))
