"""GPU parity of row-wise int8 quantisation (the "row-wise int8 quantization"
workload of Sec. IV-A) against the FP64 oracle: codes and per-row scales
must be bit-exact (integers decided by the same FP32 quotients) on every path
-- one-CTA and cluster staging (P = 2..16), the fused and split two-pass
paths, the planner's choice, host buffers and the allocation-free entry --
for FP32 and BF16 rows with ragged tails, unaligned rows, exact ties, zero
rows and rows scaled by powers of two."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def rows_input(rows, cols, seed):
    """N(0, 1) with 1% +-50 outliers, every row scaled by 2^k (k in [-20, 20]); row 0 all zero; row 1 holds
    exact ties x = s (j + 1/2) of its own scale."""
    x = synth.outliers(rows, cols, seed=seed)
    g = torch.Generator().manual_seed(seed + 1)
    k = torch.randint(-20, 21, (rows, 1), generator=g).float()
    x = x * torch.exp2(k)
    if rows > 0:
        x[0] = 0.0
    if rows > 1 and cols >= 8:
        s = 0.5  # amax 63.5 -> s = 0.5; entries s (j + 1/2) round to even
        pat = torch.tensor([63.5, 0.25, 0.75, -0.25, -0.75, 1.25, -1.75, 2.25])
        x[1] = pat.repeat(cols // 8 + 1)[:cols] * (2 * s)
    return x


def expected(x32: torch.Tensor):
    q, s = O.quant_int8(x32.numpy().astype(np.float32))
    return q, s


def run(x_dev, plan, ld_in=0, rows=None, cols=None):
    rows = x_dev.shape[0] if rows is None else rows
    cols = x_dev.shape[-1] if cols is None else cols
    q = torch.full((rows, cols), 99, dtype=torch.int8, device="cuda")
    s = torch.full((rows,), float("nan"), device="cuda")
    C.run_ex(C.QUANT_INT8, x_dev, q, plan=plan, out_dtype=C.INT8, out_scale=s, rows=rows, cols=cols, ld_in=ld_in)
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    return q.cpu().numpy(), s.cpu().numpy()


PLANS = {
    "one_cta": C.make_plan(C.PATH_ONE_CTA),
    "cluster2": C.make_plan(C.PATH_CLUSTER, 2),
    "cluster4": C.make_plan(C.PATH_CLUSTER, 4),
    "cluster8": C.make_plan(C.PATH_CLUSTER, 8),
    "cluster16": C.make_plan(C.PATH_CLUSTER, 16),
    "one_cta_tm": C.make_plan(C.PATH_ONE_CTA, retain=C.RETAIN_TMEM),
    "cluster4_tm": C.make_plan(C.PATH_CLUSTER, 4, retain=C.RETAIN_TMEM),
    "cluster16_tm": C.make_plan(C.PATH_CLUSTER, 16, retain=C.RETAIN_TMEM),
    "two_pass_g1": C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1),
    "two_pass_g3": C.make_plan(C.PATH_TWO_PASS, ctas_per_row=3),
    "auto": None,
}


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("cols", [8, 1000, 4099, 65541])
def test_quant_fp32_bit_exact(plan, cols):
    x = rows_input(67, cols, seed=cols)
    p = PLANS[plan]
    xd = x.cuda()
    if p is not None and p.path in (C.PATH_ONE_CTA, C.PATH_CLUSTER):
        q0 = torch.empty(67, cols, dtype=torch.int8, device="cuda")
        s0 = torch.empty(67, device="cuda")
        if C.plan_check(C.QUANT_INT8, xd, q0, p, out_dtype=C.INT8, out_scale=s0) != C.OK:
            # only a slice beyond one CTA's shared memory (Eq. 3) may be refused
            P = 1 if p.path == C.PATH_ONE_CTA else p.cluster_size
            cap = 131072 if p.retain == C.RETAIN_TMEM else C.slice_capacity(C.F32) * 4 - 4096
            assert -(-cols * 4 // P) > cap
            return
    q, s = run(xd, p)
    qr, sr = expected(x)
    assert np.array_equal(s.view(np.uint32), sr.view(np.uint32))
    assert np.array_equal(q, qr)
    assert (s[0] == 1.0) and (q[0] == 0).all()


@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "cluster4_tm", "two_pass_g1", "two_pass_g3"])
def test_quant_near_ties_bit_exact(plan):
    """Values within a few FP32 ulps of s (k + 1/2) for scales that are not powers of two: the codes are
    decided by the correctly rounded quotient, which a product with the reciprocal can miss by an ulp."""
    rows, cols = 24, 4096
    r = np.random.default_rng(7)
    x = np.zeros((rows, cols), dtype=np.float32)
    for i in range(rows):
        amax = np.float32(r.uniform(1.0, 2.0) * 2.0 ** r.integers(-30, 30))
        s = np.float32(amax / np.float32(127))
        k = r.integers(-127, 127, cols).astype(np.float32)
        base = (s.astype(np.float64) * (k + 0.5)).astype(np.float32)
        m = r.integers(-4, 5, cols)
        v = base.copy()
        for step in range(1, 5):  # move m ulps towards +-inf
            v = np.where(m >= step, np.nextafter(v, np.float32(np.inf)), v)
            v = np.where(-m >= step, np.nextafter(v, np.float32(-np.inf)), v)
        v = np.clip(v, -amax, amax)
        v[0] = amax
        x[i] = v
    xt = torch.from_numpy(x)
    q, sc = run(xt.cuda(), PLANS[plan])
    qr, sr = expected(xt)
    assert np.array_equal(sc, sr) and np.array_equal(q, qr)


@pytest.mark.parametrize("plan", ["one_cta", "cluster4", "two_pass_g1", "two_pass_g3"])
def test_quant_bf16_rows_and_unaligned_strides(plan):
    # BF16 rows: the oracle quantises the same values as FP32 (BF16 is a subset)
    x = synth.to_bf16(rows_input(33, 5000, seed=5))
    q, s = run(x.cuda(), PLANS[plan])
    qr, sr = expected(x.float())
    assert np.array_equal(q, qr) and np.array_equal(s, sr)
    # FP32 rows starting one element past a 16-byte boundary, with a padded stride
    cols, ld = 3001, 3007
    xb = rows_input(29, ld, seed=6)
    base = torch.zeros(29 * ld + 1, device="cuda")
    base[1:] = xb.reshape(-1).cuda()
    q2, s2 = run(base[1:], PLANS[plan], ld_in=ld, rows=29, cols=cols)
    qr2, sr2 = expected(xb[:, :cols].contiguous())
    assert np.array_equal(q2, qr2) and np.array_equal(s2, sr2)


def test_quant_many_rows_recycle_the_staged_buffers():
    x = rows_input(3000, 20000, seed=9)
    qr, sr = expected(x)
    for p in (C.make_plan(C.PATH_CLUSTER, 4), C.make_plan(C.PATH_CLUSTER, 16), C.make_plan(C.PATH_ONE_CTA),
              C.make_plan(C.PATH_CLUSTER, 2, retain=C.RETAIN_TMEM), C.make_plan(C.PATH_CLUSTER, 8, retain=C.RETAIN_TMEM)):
        q, s = run(x.cuda(), p)
        assert np.array_equal(q, qr) and np.array_equal(s, sr)


def test_quant_host_buffers_and_noalloc_match():
    x = rows_input(41, 7777, seed=12)
    qr, sr = expected(x)
    hx = x.pin_memory()
    hq = torch.empty(41, 7777, dtype=torch.int8).pin_memory()
    hs = torch.empty(41).pin_memory()
    C.run_host(C.QUANT_INT8, hx, hq, out_dtype=C.INT8, out_scale=hs)
    assert np.array_equal(hq.numpy(), qr) and np.array_equal(hs.numpy(), sr)
    xd = x.cuda()
    for _ in range(2):
        q = torch.zeros(41, 7777, dtype=torch.int8, device="cuda")
        s = torch.zeros(41, device="cuda")
        assert C.run_two_pass_noalloc(C.QUANT_INT8, xd, q, 3, out_dtype=C.INT8, out_scale=s) == C.OK
        torch.cuda.synchronize()
        assert np.array_equal(q.cpu().numpy(), qr) and np.array_equal(s.cpu().numpy(), sr)


def test_quant_refusals_launch_nothing():
    x = torch.zeros(4, 256, device="cuda")
    q = torch.zeros(4, 256, dtype=torch.int8, device="cuda")
    n0 = C.launch_count()
    assert C.run_ex_status(C.QUANT_INT8, x, q, out_dtype=C.INT8) == C.ERR_INVALID_ARG   # no scales
    assert C.run_ex_status(C.QUANT_INT8, x, x, out_dtype=C.F32, out_scale=x[0]) == C.ERR_INVALID_ARG
    assert C.launch_count() == n0
    p = C.plan(C.QUANT_INT8, 4096, 65536, C.F32, C.INT8)
    assert p.source == 3 and p.path in (C.PATH_ONE_CTA, C.PATH_CLUSTER, C.PATH_TWO_PASS)
