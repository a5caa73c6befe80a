"""GPU parity of the two-output backward ops (gradients of the weighted
variance and of the Pearson correlation of a row pair) against the FP64
oracle, through the C ABI (credit_run_bwd with dx2): every path on rows with
a ragged tail, unaligned rows on the two-pass path, and the refusals.  The
bound is in parity_util.pair_error."""
import pytest
import torch

from paper_2609_01864_gb300 import credit as C

import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield
    torch.cuda.synchronize()


def check(op, dtype, rows, cols, ld, plan, seed=0):
    x, d, g = U.pair_inputs(op, dtype, rows, cols, ld=ld, seed=seed)
    gx, gd = x.cuda(), d.cuda()
    o1 = torch.full_like(gx, float("nan"))
    o2 = torch.full_like(gx, float("nan"))
    C.run_bwd(op, gx, gd, o1, plan=plan, rows=rows, cols=cols, ld=ld, scale=g.cuda(), dx2=o2)
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    r1, r2 = U.pair_reference(op, x, d, g, cols)
    err = U.pair_error(op, dtype, U.to64(o1)[:, :cols], U.to64(o2)[:, :cols], r1, r2, x, d, g, cols)
    assert err <= 1.0, err
    if ld > cols:
        assert torch.isnan(o1[:, cols:].float()).all() and torch.isnan(o2[:, cols:].float()).all()


PLANS = {
    "two_pass_g1": (C.make_plan(C.PATH_TWO_PASS, ctas_per_row=1), 70001),
    "two_pass_g3": (C.make_plan(C.PATH_TWO_PASS, ctas_per_row=3), 70001),
    "one_cta": (C.make_plan(C.PATH_ONE_CTA), 5003),
    "cluster4": (C.make_plan(C.PATH_CLUSTER, 4), 70001),
    "cluster16": (C.make_plan(C.PATH_CLUSTER, 16), 70001),
    "auto": (None, 70001),
}


@pytest.mark.parametrize("plan", list(PLANS))
@pytest.mark.parametrize("dtype", [C.F32, C.BF16], ids=["f32", "bf16"])
@pytest.mark.parametrize("op", [C.WVAR_BWD, C.PEARSON_BWD], ids=["wvar", "pearson"])
def test_pair_matches_oracle(op, dtype, plan):
    p, cols = PLANS[plan]
    ld = -(-cols // 8) * 8 + 8
    check(op, dtype, 29, cols, ld, p, seed=op + dtype)


@pytest.mark.parametrize("op", [C.WVAR_BWD, C.PEARSON_BWD], ids=["wvar", "pearson"])
def test_pair_unaligned_rows_and_many_rows(op):
    check(op, C.F32, 17, 4099, 0, None, seed=3)                                   # two-pass fallback
    check(op, C.F32, 700, 8195, 8196, C.make_plan(C.PATH_CLUSTER, 4), seed=4)     # rows recycle buffers


def test_pair_refusals_launch_nothing():
    x = torch.zeros(8, 4096, device="cuda")
    n0 = C.launch_count()
    assert C.run_bwd_status(C.WVAR_BWD, x, x, x) == C.ERR_INVALID_ARG                 # no dx2
    assert C.run_bwd_status(C.PEARSON_BWD, x, x, x) == C.ERR_INVALID_ARG
    assert C.launch_count() == n0
