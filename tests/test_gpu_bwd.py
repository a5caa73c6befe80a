"""GPU parity of the backward ops (dx of softmax, LayerNorm, RMSNorm; dz of
softmax and of the cross entropy from logits) against the FP64 oracle,
through the C ABI (credit_run_bwd).

Every path (fused and split two-pass, one-CTA, clusters of 2-16) on rows
that span several groups per thread and end in a ragged tail; many rows per
cluster (row buffers, exchange slots and mbarrier phases recycled); single
and double buffering (bitwise equal); tiny rows with empty slices; in-place
dx; unaligned rows (two-pass only); the refusals; determinism; and sampled
rows of full-size (4096 x 262144) calls.  The bound is in parity_util.bwd_error.
"""
import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C

import parity_util as U

pytestmark = pytest.mark.gpu

OPS = [C.SOFTMAX_BWD, C.LAYERNORM_BWD, C.RMSNORM_BWD, C.SOFTMAX_LOGITS_BWD, C.XENT_BWD]
IDS = ["softmax", "layernorm", "rmsnorm", "softmax_logits", "xent"]
DTYPES = [C.F32, C.BF16]


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def pad(cols, dtype):
    v = 4 if dtype == C.F32 else 8
    return -(-cols // v) * v


def run(op, dtype, a, dy, gamma, mean, rstd, rows, cols, ld=0, plan=None, dx=None):
    d = lambda t: None if t is None else t.cuda()  # noqa: E731
    ga, gdy = a.cuda(), dy.cuda()
    out = torch.full_like(ga, float("nan")) if dx is None else dx
    if op == C.XENT_BWD:  # the last input is the per-row scale
        C.run_bwd(op, ga, gdy, out, plan=plan, rows=rows, cols=cols, ld=ld, scale=d(rstd))
    else:
        C.run_bwd(op, ga, gdy, out, plan=plan, rows=rows, cols=cols, ld=ld, gamma=d(gamma), mean=d(mean),
                  rstd=d(rstd))
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    return out


def check(op, dtype, rows, cols, ld, plan, seed=0):
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, ld=ld, seed=seed)
    out = run(op, dtype, a, dy, g, m, r, rows, cols, ld, plan)
    ref = U.bwd_reference(op, dtype, a, dy, g, m, r, rows, cols, ld)
    err = U.bwd_error(op, dtype, U.to64(out)[:, :cols], ref, a, dy, g, m, r, cols)
    assert err <= 1.0, err
    if ld > cols:  # the padding is not written
        assert torch.isnan(out[:, cols:].float()).all()
    return out


PLANS = {
    "two_pass_g1": (C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1), 70001),
    "two_pass_g3": (C.make_plan(C.PATH_TWO_PASS, ctas_per_row=3), 70001),
    "one_cta": (C.make_plan(C.PATH_ONE_CTA), 5003),
    "cluster2": (C.make_plan(C.PATH_CLUSTER, 2), 20011),
    "cluster4": (C.make_plan(C.PATH_CLUSTER, 4), 70001),
    "cluster8": (C.make_plan(C.PATH_CLUSTER, 8), 70001),
    "cluster16": (C.make_plan(C.PATH_CLUSTER, 16), 70001),
    "auto": (None, 70001),
}


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "bf16"])
@pytest.mark.parametrize("op", OPS, ids=IDS)
def test_bwd_matches_oracle(op, dtype, plan):
    p, cols = PLANS[plan]
    check(op, dtype, 37, cols, pad(cols, dtype) + (8 if dtype == C.F32 else 0), p, seed=op + dtype)


@pytest.mark.parametrize("op", OPS, ids=IDS)
def test_unaligned_rows_run_two_pass(op):
    # contiguous rows of 4099 FP32: every row after the first starts off the 16-byte grid
    for plan in (None, C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1), C.make_plan(C.PATH_TWO_PASS, ctas_per_row=4)):
        check(op, C.F32, 21, 4099, 0, plan, seed=7)


@pytest.mark.parametrize("op", OPS, ids=IDS)
def test_many_rows_recycle_buffers_and_slots(op):
    # far more rows than resident clusters: every row buffer, exchange slot and mbarrier phase is reused
    for P in (1, 4, 16):
        plan = C.make_plan(C.PATH_ONE_CTA) if P == 1 else C.make_plan(C.PATH_CLUSTER, P)
        check(op, C.F32, 1500, 8195, 8196, plan, seed=11 + P)


@pytest.mark.parametrize("op", OPS, ids=IDS)
def test_single_buffer_refilled_chunk_by_chunk(op):
    # 64 KiB slices at P = 16: only one row buffer fits, refilled in 8 chunks behind the write pass
    check(op, C.F32, 300, 262147, 262148, C.make_plan(C.PATH_CLUSTER, 16), seed=17)
    check(op, C.BF16, 200, 300007, 300008, C.make_plan(C.PATH_CLUSTER, 16, ring_chunks=1), seed=19)


def test_single_and_double_buffering_agree_bitwise():
    op, dtype, rows, cols = C.LAYERNORM_BWD, C.F32, 300, 40000
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, seed=3)
    outs = []
    for nbuf in (1, 2):
        outs.append(run(op, dtype, a, dy, g, m, r, rows, cols, 0, C.make_plan(C.PATH_CLUSTER, 8, ring_chunks=nbuf)))
    assert torch.equal(outs[0], outs[1])
    ref = U.bwd_reference(op, dtype, a, dy, g, m, r, rows, cols)
    assert U.bwd_error(op, dtype, U.to64(outs[0]), ref, a, dy, g, m, r, cols) <= 1.0


@pytest.mark.parametrize("cols", [1, 3, 17, 64])
@pytest.mark.parametrize("op", OPS, ids=IDS)
def test_tiny_rows_and_empty_slices(op, cols):
    for plan in (C.make_plan(C.PATH_CLUSTER, 16), C.make_plan(C.PATH_ONE_CTA), None):
        check(op, C.F32, 5, cols, pad(cols, C.F32), plan, seed=cols)


@pytest.mark.parametrize("dtype", DTYPES, ids=["f32", "bf16"])
def test_gamma_staged_or_loaded_gives_the_same_bits(dtype):
    op, rows, cols = C.LAYERNORM_BWD, 200, 30000
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, seed=13)
    plan = C.make_plan(C.PATH_CLUSTER, 4)
    staged = run(op, dtype, a, dy, g, m, r, rows, cols, 0, plan)
    buf = torch.empty(cols + 1, device="cuda")
    buf[1:] = g.cuda()
    loaded = run(op, dtype, a, dy, buf[1:], m, r, rows, cols, 0, plan)  # gamma off the 16-byte grid: L2 loads
    assert torch.equal(staged, loaded)


def test_in_place_matches_out_of_place():
    op, dtype, rows, cols = C.RMSNORM_BWD, C.BF16, 64, 65536
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, seed=5)
    for plan in (C.make_plan(C.PATH_CLUSTER, 4), C.make_plan(C.PATH_TWO_PASS, ctas_per_row=2),
                 C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1)):
        ref = run(op, dtype, a, dy, g, m, r, rows, cols, 0, plan)
        gdy = dy.cuda()
        run(op, dtype, a, gdy, g, m, r, rows, cols, 0, plan, dx=gdy)  # dx written over dy
        assert torch.equal(gdy, ref)


def test_deterministic_and_paths_agree():
    op, dtype, rows, cols = C.SOFTMAX_BWD, C.F32, 128, 131072
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, seed=9)
    p8 = C.make_plan(C.PATH_CLUSTER, 8)
    o1 = run(op, dtype, a, dy, g, m, r, rows, cols, 0, p8)
    o2 = run(op, dtype, a, dy, g, m, r, rows, cols, 0, p8)
    assert torch.equal(o1, o2)
    ref = U.bwd_reference(op, dtype, a, dy, g, m, r, rows, cols)
    for plan in (C.make_plan(C.PATH_CLUSTER, 16), C.make_plan(C.PATH_TWO_PASS, ctas_per_row=2)):
        o = run(op, dtype, a, dy, g, m, r, rows, cols, 0, plan)
        assert U.bwd_error(op, dtype, U.to64(o), ref, a, dy, g, m, r, cols) <= 1.0


def test_refusals_launch_nothing():
    x = torch.zeros(8, 4099, device="cuda")
    rs = torch.ones(8, device="cuda")
    n0 = C.launch_count()
    st = C.run_bwd_status
    # staged paths need 16-byte aligned rows
    assert st(C.RMSNORM_BWD, x, x, x, rstd=rs, plan=C.make_plan(C.PATH_CLUSTER, 4)) == C.ERR_UNSUPPORTED
    y = torch.zeros(8, 70000, device="cuda")
    assert st(C.RMSNORM_BWD, y, y, y, rstd=rs, plan=C.make_plan(C.PATH_ONE_CTA)) == C.ERR_UNSUPPORTED  # Eq. 3
    assert st(C.RMSNORM_BWD, y, y, y, rstd=rs, plan=C.make_plan(C.PATH_CLUSTER, 3)) == C.ERR_UNSUPPORTED
    assert st(C.RMSNORM_BWD, y, y, y, rstd=rs,
              plan=C.make_plan(C.PATH_CLUSTER, 8, fill_share=0.2)) == C.ERR_UNSUPPORTED
    assert st(C.RMSNORM_BWD, y, y, y, rstd=rs, plan=C.make_plan(C.PATH_CLUSTER, 8, ring_chunks=3)) == C.ERR_UNSUPPORTED
    assert st(C.LAYERNORM_BWD, y, y, y, rstd=rs) == C.ERR_INVALID_ARG          # no mean
    assert st(C.RMSNORM_BWD, y, y, y) == C.ERR_INVALID_ARG                     # no rstd
    assert st(C.LOGSUMEXP, y, y, y) == C.ERR_INVALID_ARG                       # not a backward op
    q = torch.zeros(8, 64, device="cuda", dtype=torch.float8_e4m3fn)
    assert st(C.SOFTMAX_BWD, q, q, q) == C.ERR_UNSUPPORTED
    assert C.launch_count() == n0
    assert st(C.SOFTMAX_BWD, y, y, y, rows=0, cols=70000) == C.OK
    assert C.launch_count() == n0


def test_planner_choices():
    narrow = C.plan_bwd(C.LAYERNORM_BWD, 4096, 2048, C.F32)
    assert (narrow.path, narrow.ctas_per_row) == (C.PATH_TWO_PASS, 1)
    for cols in (16384, 65536, 131072):  # two row buffers of a and dy plus gamma fit at P = 2, 8, 16
        p = C.plan_bwd(C.RMSNORM_BWD, 4096, cols, C.F32)
        assert p.path == C.PATH_CLUSTER and p.ring_chunks == 2 and p.smem_bytes > 0
        x = torch.zeros(4, cols, device="cuda")
        g = torch.ones(cols, device="cuda")
        assert C.bwd_plan_check(C.RMSNORM_BWD, x, x, x, p, gamma=g, rstd=torch.ones(4, device="cuda")) == C.OK
    assert C.plan_bwd(C.RMSNORM_BWD, 4096, 262144, C.F32).path == C.PATH_TWO_PASS  # only a single buffer fits
    wide = C.plan_bwd(C.SOFTMAX_BWD, 64, 1 << 21, C.F32)
    assert wide.path == C.PATH_TWO_PASS and wide.ctas_per_row > 1


@pytest.mark.parametrize("op,dtype", [(C.LAYERNORM_BWD, C.F32), (C.SOFTMAX_BWD, C.BF16), (C.RMSNORM_BWD, C.F32)])
def test_full_size_sampled_rows(op, dtype):
    rows, cols = 4096, 262144
    a, dy, g, m, r = U.bwd_inputs(op, dtype, rows, cols, seed=21, device="cuda")
    out = run(op, dtype, a, dy, g, m, r, rows, cols)
    pick = [0, 1, 1000, 2047, 4094, 4095]
    sub = lambda t: None if t is None else t[pick].cpu()  # noqa: E731
    g = None if g is None else g.cpu()
    ref = U.bwd_reference(op, dtype, sub(a), sub(dy), g, sub(m), sub(r), len(pick), cols)
    assert U.bwd_error(op, dtype, U.to64(out[pick]), ref, sub(a), sub(dy), g, sub(m), sub(r), cols) <= 1.0
