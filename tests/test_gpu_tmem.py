"""GPU parity of the staged paths with the slice retained in tensor memory.

Forced RETAIN_TMEM plans of every cluster size against the FP64 oracle, over
shapes that span several 16 KiB chunks, ragged tails, rows that start off the
16-byte grid, slices up to the 128 KiB TMEM capacity and more rows than
persistent clusters (so both TMEM row buffers and all four exchange slots are
recycled); the three gamma / beta modes (resident, streamed, direct); the
refusals (slice over capacity, logsumexp, FP8-output norms); agreement with
the shared-memory ring kernel; and run-to-run bitwise determinism.
"""
import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C

import parity_util as U

pytestmark = pytest.mark.gpu

TM_CAP = 8 * 16384  # input bytes of one retained slice


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def tm_plan(P):
    return C.make_plan(C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER, P, retain=C.RETAIN_TMEM)


def fits(cols, isz, P):
    groups = (cols * isz) // 16
    return -(-groups // P) * 16 <= TM_CAP


def affine(op, cols, seed=3):
    from paper_2609_01864_gb300 import synth
    if op in (C.LAYERNORM, C.RMSNORM):
        g, b = synth.gamma_beta(cols, seed=seed)
        return g, (b if op == C.LAYERNORM else None)
    return None, None


TM_OPS = [C.SOFTMAX, C.LAYERNORM, C.RMSNORM]


@pytest.mark.parametrize("P", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("op", TM_OPS)
@pytest.mark.parametrize("rows,cols", [(3, 1), (9, 17), (200, 4099), (37, 16385), (64, 70001)])
def test_fp32_tmem_matches_oracle(op, P, rows, cols):
    if not fits(cols, 4, P):
        pytest.skip("slice over the TMEM capacity (refusal tested separately)")
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers" if op != C.SOFTMAX else "normal", std=3.0,
                        seed=rows * 31 + cols + P)
    g, b = affine(op, cols)
    U.check_against_oracle(op, x, None, plan=tm_plan(P), gamma=g, beta=b)


@pytest.mark.parametrize("P", [16])
@pytest.mark.parametrize("op", TM_OPS)
def test_full_capacity_slice(op, P):
    # 524288 FP32 columns over 16 CTAs: exactly 128 KiB (8 chunks) per CTA
    rows, cols = 24, 524288
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers" if op != C.SOFTMAX else "normal", std=3.0, seed=77)
    g, b = affine(op, cols)
    U.check_against_oracle(op, x, None, plan=tm_plan(P), gamma=g, beta=b)


DTYPES = [(C.BF16, C.BF16), (C.F32, C.BF16), (C.BF16, C.F32), (C.FP8_E4M3, C.F32), (C.FP8_E4M3, C.BF16)]


@pytest.mark.parametrize("P", [1, 4, 16])
@pytest.mark.parametrize("op", TM_OPS)
@pytest.mark.parametrize("dt", DTYPES, ids=lambda d: f"{d[0]}to{d[1]}")
@pytest.mark.parametrize("rows,cols", [(40, 2053), (21, 40007)])
def test_low_precision_tmem_matches_oracle(op, P, dt, rows, cols):
    tin, tout = dt
    isz = {C.F32: 4, C.BF16: 2, C.FP8_E4M3: 1}[tin]
    if not fits(cols, isz, P):
        pytest.skip("slice over the TMEM capacity")
    x, s = U.make_input(tin, rows, cols, kind="outliers" if op != C.SOFTMAX else "normal", std=3.0,
                        seed=cols + tin * 13 + tout + P)
    g, b = affine(op, cols)
    U.check_against_oracle(op, x, s, out_dtype=tout, plan=tm_plan(P), gamma=g, beta=b)


@pytest.mark.parametrize("P", [1, 8])
@pytest.mark.parametrize("dt", [C.F32, C.BF16, C.FP8_E4M3])
def test_softmax_fp8_output(dt, P):
    x, s = U.make_input(dt, 30, 20011, std=3.0, seed=dt + P)
    U.check_against_oracle(C.SOFTMAX, x, s, out_dtype=C.FP8_E4M3, plan=tm_plan(P))


@pytest.mark.parametrize("mode", ["resident", "stream", "direct"])
@pytest.mark.parametrize("op", [C.LAYERNORM, C.RMSNORM])
@pytest.mark.parametrize("dt,cols,P", [(C.F32, 16384, 1), (C.F32, 65536, 4), (C.F32, 262144, 8),
                                       (C.BF16, 40000, 2), (C.FP8_E4M3, 65536, 1)])
def test_affine_modes(op, dt, cols, P, mode, monkeypatch):
    if mode != "resident":
        monkeypatch.setenv("CREDIT_TM_AFFINE", mode)
    rows = 48
    x, s = U.make_input(dt, rows, cols, kind="outliers", seed=cols + P + len(mode))
    g, b = affine(op, cols, seed=9)
    U.check_against_oracle(op, x, s, out_dtype=C.F32 if dt == C.FP8_E4M3 else dt, plan=tm_plan(P), gamma=g, beta=b)


def test_layernorm_with_affine_from_l2_repeats_exactly(monkeypatch):
    """LayerNorm whose gamma / beta the tensor-memory kernel would read from L2 runs on the shared-memory ring,
    also under an explicit tensor-memory plan (the tensor-memory kernel returned wrong rows on that
    combination in soak runs): 48 x 262144 FP32 at P = 8, within the oracle's bound, then 30 more calls into
    NaN-filled outputs, each bit-identical to the first."""
    monkeypatch.setenv("CREDIT_TM_AFFINE", "direct")
    rows, cols, P = 48, 262144, 8
    x, s = U.make_input(C.F32, rows, cols, kind="outliers", seed=cols + P)
    g, b = affine(C.LAYERNORM, cols, seed=9)
    _, first = U.check_against_oracle(C.LAYERNORM, x, s, plan=tm_plan(P), gamma=g, beta=b)
    xd, gd, bd = x.cuda(), g.cuda(), b.cuda()
    out = torch.empty_like(xd)
    for _ in range(30):
        out.fill_(float("nan"))
        C.run_ex(C.LAYERNORM, xd, out, plan=tm_plan(P), gamma=gd, beta=bd)
        torch.cuda.synchronize()
        assert torch.equal(out, first)
    assert C.device_error() == C.OK


@pytest.mark.parametrize("P", [1, 4])
@pytest.mark.parametrize("op", TM_OPS)
def test_unaligned_rows_and_strides(op, P):
    rows, cols, ld = 6, 3001, 3011
    dt = C.BF16
    base, _ = U.make_input(dt, rows, ld + 8, std=2.0, seed=5)
    dev = base.cuda()
    view_ptr = dev.view(-1).data_ptr() + 3 * 2  # rows start 6 bytes off the 16-byte grid
    x_cpu = torch.stack([base.view(-1)[3 + r * ld: 3 + r * ld + cols] for r in range(rows)])
    out_buf = torch.empty(rows * ld + 16, device="cuda", dtype=torch.float32)
    out_ptr = out_buf.data_ptr() + 4 * 4
    g, b = affine(op, cols)
    gd = None if g is None else g.cuda()
    bd = None if b is None else b.cuda()
    C.run_ex(op, view_ptr, out_ptr, rows=rows, cols=cols, in_dtype=dt, out_dtype=C.F32, ld_in=ld, ld_out=ld,
             gamma=gd, beta=bd, plan=tm_plan(P))
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    y = torch.stack([out_buf[4 + r * ld: 4 + r * ld + cols] for r in range(rows)]).double().cpu().numpy()
    ref = U.reference(op, dt, x_cpu, None, g, b)
    assert U.error_metric(op, C.F32, y, ref) <= 1.0


def test_refusals_launch_nothing():
    x = torch.randn(4, 1 << 20, device="cuda")  # 4 MiB rows: 256 KiB slices at P = 16
    y = torch.empty_like(x)
    n0 = C.launch_count()
    for op in TM_OPS:
        assert C.run_ex_status(op, x, y, plan=tm_plan(16)) == C.ERR_UNSUPPORTED
    xs = torch.randn(4, 4096, device="cuda")
    lse = torch.empty(4, device="cuda")
    assert C.run_ex_status(C.LOGSUMEXP, xs, lse, plan=tm_plan(1)) == C.ERR_UNSUPPORTED
    y8 = torch.empty(4, 4096, device="cuda", dtype=torch.float8_e4m3fn)
    osc = torch.empty(4, device="cuda")
    assert C.run_ex_status(C.RMSNORM, xs, y8, plan=tm_plan(1), out_dtype=C.FP8_E4M3,
                           out_scale=osc) == C.ERR_UNSUPPORTED
    assert C.launch_count() == n0


@pytest.mark.parametrize("P", [1, 8])
@pytest.mark.parametrize("op", TM_OPS)
def test_agrees_with_shared_memory_ring(op, P):
    # same slicing, chunking and h; the two kernels differ only in how the
    # partials are merged (CTA tree + fixed-order combine vs warp partials +
    # one 32-lane tree), so they agree to the FP32 bound
    rows, cols = 50, (32768 if P == 1 else 131072)  # 128 / 64 KiB slices: legal for both kernels
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers", std=2.0, seed=21 + P)
    g, b = affine(op, cols)
    path = C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER
    smem_plan = C.make_plan(path, P, retain=C.RETAIN_SMEM)
    o1, _ = U.run_gpu(op, x, None, plan=tm_plan(P), gamma=g, beta=b)
    o2, _ = U.run_gpu(op, x, None, plan=smem_plan, gamma=g, beta=b)
    torch.cuda.synchronize()
    assert o1 is not None and o2 is not None
    assert U.error_metric(op, C.F32, U.to64(o1), U.to64(o2)) <= 1.0


def test_deterministic_and_auto_policy(monkeypatch):
    x, _ = U.make_input(C.F32, 33, 12345, std=2.0, seed=11)
    o1, _ = U.run_gpu(C.SOFTMAX, x, None, plan=tm_plan(8))
    o2, _ = U.run_gpu(C.SOFTMAX, x, None, plan=tm_plan(8))
    monkeypatch.setenv("CREDIT_RETAIN", "tmem")
    o3, _ = U.run_gpu(C.SOFTMAX, x, None, plan=C.make_plan(C.PATH_CLUSTER, 8))
    torch.cuda.synchronize()
    assert torch.equal(o1, o2) and torch.equal(o1, o3)
