"""GPU parity: every path of every op against the FP64 oracle, through the C ABI.

Sizes are small enough for the oracle to finish in well under a second per
case but span several 16 KiB staging chunks, several CTAs per row and ragged
tails (cols not a multiple of the 16-byte group, rows that start off the
16-byte grid).
"""
import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

import parity_util as U

pytestmark = pytest.mark.gpu

OPS = [C.SOFTMAX, C.LOGSUMEXP, C.LAYERNORM, C.RMSNORM]
PLANS = {
    "one_cta": C.make_plan(C.PATH_ONE_CTA),
    "cluster2": C.make_plan(C.PATH_CLUSTER, 2),
    "cluster4": C.make_plan(C.PATH_CLUSTER, 4),
    "cluster8": C.make_plan(C.PATH_CLUSTER, 8),
    "cluster16": C.make_plan(C.PATH_CLUSTER, 16),
    "two_pass_g1": C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1),
    "two_pass_g5": C.make_plan(C.PATH_TWO_PASS, ctas_per_row=5),
}


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def _affine(op, cols, seed=1):
    if op in (C.LAYERNORM, C.RMSNORM):
        g, b = synth.gamma_beta(cols, seed=seed)
        return g, (b if op == C.LAYERNORM else None)
    return None, None


# --------------------------------------------------------------- FP32, shapes x paths
@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("rows,cols", [(3, 1), (5, 3), (9, 17), (6, 1000), (4, 4099), (3, 70001)])
def test_fp32_paths_match_oracle(op, plan, rows, cols):
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers" if op in (C.LAYERNORM, C.RMSNORM) else "normal",
                        std=3.0, seed=rows * 7919 + cols)
    g, b = _affine(op, cols)
    U.check_against_oracle(op, x, None, plan=PLANS[plan], gamma=g, beta=b)


# --------------------------------------------------------------- dtypes x paths
DTYPES = [(C.BF16, C.BF16), (C.FP8_E4M3, C.FP8_E4M3), (C.F32, C.BF16), (C.F32, C.FP8_E4M3),
          (C.BF16, C.F32), (C.FP8_E4M3, C.F32)]


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("op", OPS)
@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: f"{d[0]}to{d[1]}")
@pytest.mark.parametrize("rows,cols", [(5, 2053), (3, 40007)])
def test_low_precision_paths_match_oracle(op, plan, dt, rows, cols):
    tin, tout = dt
    if op == C.LOGSUMEXP and tout != C.F32:
        tout = C.F32
    x, s = U.make_input(tin, rows, cols, kind="outliers" if op in (C.LAYERNORM, C.RMSNORM) else "normal",
                        std=3.0, seed=cols + tin * 13 + tout)
    g, b = _affine(op, cols)
    U.check_against_oracle(op, x, s, out_dtype=tout, plan=PLANS[plan], gamma=g, beta=b)


@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "two_pass_g1", "two_pass_g5"])
@pytest.mark.parametrize("op", [C.SOFTMAX, C.LOGSUMEXP])
@pytest.mark.parametrize("tout", [C.FP8_E4M3, C.F32])
def test_fp8_rows_with_negative_and_zero_scales(op, plan, tout):
    """E4M3 rows whose per-row scale is negative (x = scale * code flips the order of the codes), zero
    (every x is 0: the uniform distribution), tiny or large, with codes spanning the whole E4M3 range
    (+-448, subnormals, +-0): the softmax statistics and the FP8 output codes against the oracle."""
    if op == C.LOGSUMEXP:
        tout = C.F32
    rows, cols = 12, 20011
    g = torch.Generator().manual_seed(21)
    codes = torch.randint(0, 256, (rows, cols), generator=g, dtype=torch.int16)
    codes = torch.where((codes & 0x7F) == 0x7F, codes - 1, codes).to(torch.uint8)  # no NaN codes
    codes[:, 0] = 0x7E   # +448
    codes[:, 1] = 0xFE   # -448
    codes[:, 2] = 0x01   # smallest subnormal
    codes[:, 3] = 0x80   # -0
    x = codes.view(torch.float8_e4m3fn)
    sc = torch.tensor([-1.0, 0.0, 1e-3, -1e-3, 0.25, -0.25, 0.05, -0.02, 2.0 ** -20, -(2.0 ** -20), 0.01, -0.5],
                      dtype=torch.float32)
    if op == C.SOFTMAX and tout == C.F32:
        sc = sc.clamp(-0.05, 0.05)  # |x - max| <= 45: every probability a normal FP32 number
    U.check_against_oracle(op, x, sc, out_dtype=tout, plan=PLANS[plan])


@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "two_pass_g1", "two_pass_g5"])
@pytest.mark.parametrize("op,tout", [(C.SOFTMAX, C.FP8_E4M3), (C.SOFTMAX, C.F32), (C.LOGSUMEXP, C.F32)])
def test_fp8_rows_whose_maximum_lies_below_the_scale_bound(op, tout, plan):
    """E4M3 rows whose codes do not reach +-448 in the direction of their scale, so the row maximum lies below
    |scale| * 448: far below (every term about that bound underflows; sign folded or not; a constant row) and
    a little below (the terms about the bound are kept and rescaled to the row maximum).  Row lengths off the
    16-byte grid give head and tail elements."""
    rows, cols = 8, 20011
    spec = [  # (lowest code, highest code, scale)
        (0x80, 0xFE, 0.1),     # values -448..-0: x in [-44.8, 0]
        (0x00, 0x60, 0.05),    # 0..32: max 1.6 against the bound 22.4
        (0x00, 0x70, 0.01),    # 0..128: max 1.28 against 4.48
        (0x00, 0x7E, -0.1),    # 0..448 with a negative scale: x in [-44.8, 0]
        (0x80, 0xFE, -0.002),  # -448..-0 with a negative scale: the maximum is the bound
        (0x38, 0x48, 0.5),     # 1..4: x in [0.5, 2] against 224
        (0x40, 0x40, 0.3),     # one code: the uniform distribution
        (0x00, 0x68, 0.02),    # 0..64: max 1.28 against 8.96
    ]
    g = torch.Generator().manual_seed(33)
    codes = torch.empty(rows, cols, dtype=torch.uint8)
    for r, (lo, hi, _) in enumerate(spec):
        codes[r] = torch.randint(lo, hi + 1, (cols,), generator=g, dtype=torch.int16).to(torch.uint8)
    x = codes.view(torch.float8_e4m3fn)
    sc = torch.tensor([s for _, _, s in spec], dtype=torch.float32)
    U.check_against_oracle(op, x, sc, out_dtype=tout, plan=PLANS[plan])


# --------------------------------------------------------------- config 1
@pytest.mark.parametrize("plan", ["one_cta", "cluster4"])
def test_softmax_256x4096_fp32_one_cta_and_cluster4(plan):
    x, _ = U.make_input(C.F32, 256, 4096, seed=synth.SEED_DATA)
    m, out = U.check_against_oracle(C.SOFTMAX, x, None, plan=PLANS[plan])
    sums = out.double().sum(dim=1).cpu().numpy()
    assert np.max(np.abs(sums - 1.0)) <= 1e-5


# --------------------------------------------------------------- layouts and edges
@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "two_pass_g1", "two_pass_g5"])
@pytest.mark.parametrize("op", OPS)
def test_unaligned_rows_and_strides(op, plan):
    rows, cols, ld = 6, 3001, 3011
    dt = C.BF16
    base, _ = U.make_input(dt, rows, ld + 8, std=2.0, seed=5)
    dev = base.cuda()
    # rows start 3 elements into the buffer (6 bytes: off the 16-byte grid), stride ld
    flat = dev.view(-1)
    view_ptr = flat.data_ptr() + 3 * 2
    x_cpu = torch.stack([base.view(-1)[3 + r * ld: 3 + r * ld + cols] for r in range(rows)])
    out_buf = torch.empty(rows * ld + 16, device="cuda", dtype=torch.float32)
    out_ptr = out_buf.data_ptr() + 4 * 4  # 16-byte aligned start, FP32 out
    g, b = _affine(op, cols)
    gd = None if g is None else g.cuda()
    bd = None if b is None else b.cuda()
    C.run_ex(op, view_ptr, out_ptr, rows=rows, cols=cols, in_dtype=dt, out_dtype=C.F32, ld_in=ld,
             ld_out=0 if op == C.LOGSUMEXP else ld, gamma=gd, beta=bd, plan=PLANS[plan])
    torch.cuda.synchronize()
    if op == C.LOGSUMEXP:
        y = out_buf[4:4 + rows].double().cpu().numpy()
    else:
        y = torch.stack([out_buf[4 + r * ld: 4 + r * ld + cols] for r in range(rows)]).double().cpu().numpy()
    ref = U.reference(op, dt, x_cpu, None, g, b)
    assert U.error_metric(op, C.F32, y, ref) <= 1.0


@pytest.mark.parametrize("plan", ["one_cta", "cluster8", "two_pass_g1", "two_pass_g5"])
@pytest.mark.parametrize("op", OPS)
def test_deterministic_bitwise(op, plan):
    x, _ = U.make_input(C.F32, 17, 12345, std=2.0, seed=11)
    o1, _ = U.run_gpu(op, x, None, plan=PLANS[plan])
    o2, _ = U.run_gpu(op, x, None, plan=PLANS[plan])
    torch.cuda.synchronize()
    assert torch.equal(o1, o2)


@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "two_pass_g1", "two_pass_g5"])
def test_in_place(plan):
    x, _ = U.make_input(C.F32, 8, 5000, std=2.0, seed=12)
    ref = U.reference(C.SOFTMAX, C.F32, x)
    d = x.cuda()
    C.run_ex(C.SOFTMAX, d, d, plan=PLANS[plan])
    torch.cuda.synchronize()
    assert U.error_metric(C.SOFTMAX, C.F32, U.to64(d), ref) <= 1.0


def test_zero_rows_is_a_noop_and_bad_plans_are_rejected():
    x = torch.zeros(0, 64, device="cuda")
    assert C.run_ex(C.SOFTMAX, x, x, rows=0, cols=64) == C.OK
    x = torch.randn(4, 1 << 20, device="cuda")
    y = torch.empty_like(x)
    # one CTA cannot stage a 4 MiB row (Eq. 3): rejected, nothing launched
    n0 = C.launch_count()
    assert C.run_ex_status(C.SOFTMAX, x, y, plan=C.make_plan(C.PATH_ONE_CTA)) == C.ERR_UNSUPPORTED
    assert C.run_ex_status(C.SOFTMAX, x, y, plan=C.make_plan(C.PATH_CLUSTER, 2)) == C.ERR_UNSUPPORTED
    assert C.run_ex_status(C.SOFTMAX, x, y, plan=C.make_plan(C.PATH_CLUSTER, 17)) == C.ERR_UNSUPPORTED
    assert C.run_ex_status(C.SOFTMAX, x, y, plan=C.make_plan(C.PATH_TWO_PASS, ctas_per_row=0)) == C.ERR_UNSUPPORTED
    assert C.launch_count() == n0


def test_simple_entry_points_use_the_planner():
    x, _ = U.make_input(C.F32, 64, 8192, std=2.0, seed=13)
    d = x.cuda()
    for op, fn in ((C.SOFTMAX, C.softmax), (C.LOGSUMEXP, C.logsumexp), (C.LAYERNORM, C.layernorm),
                   (C.RMSNORM, C.rmsnorm)):
        y = fn(d)
        torch.cuda.synchronize()
        ref = U.reference(op, C.F32, x)
        assert U.error_metric(op, C.F32, U.to64(y), ref) <= 1.0
    xb = d.to(torch.bfloat16)
    yb = C.softmax(xb)
    torch.cuda.synchronize()
    ref = U.reference(C.SOFTMAX, C.BF16, xb.cpu())
    assert U.error_metric(C.SOFTMAX, C.BF16, U.to64(yb), ref) <= 1.0


# --------------------------------------------------------------- gamma/beta staging modes
# 16-byte-aligned rows with gamma/beta: the ring kernel stages gamma/beta in
# shared memory, resident for small slices and streamed for wide ones; more
# rows than persistent clusters make every CTA recycle its rings.
@pytest.mark.parametrize("op", [C.LAYERNORM, C.RMSNORM])
@pytest.mark.parametrize("dt,cols,P", [(C.F32, 4096, 1), (C.F32, 16384, 2), (C.F32, 40000, 1), (C.F32, 65536, 4),
                                       (C.BF16, 8192, 1), (C.BF16, 40000, 2), (C.FP8_E4M3, 65536, 1)])
def test_affine_staging_modes(op, dt, cols, P):
    rows = 400
    x, s = U.make_input(dt, rows, cols, kind="outliers", seed=cols + P)
    g, b = _affine(op, cols, seed=7)
    plan = C.make_plan(C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER, P)
    U.check_against_oracle(op, x, s, plan=plan, gamma=g, beta=b)
