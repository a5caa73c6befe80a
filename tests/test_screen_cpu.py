"""The structural screen of the profitability model (Sec. III-D, last
paragraph; the negative controls of Sec. IV-C), pure host code: the four
reduction-reuse ops and the int8 quantiser are candidates; log-sum-exp (no
reread), the stencil (no reduction stage), the scan (ordered carries, K
grows with P) and selection (remote state growing with N) are rejected
before any clustered code runs."""
import pytest

from paper_2609_01864_gb300 import build as B
from paper_2609_01864_gb300 import credit as C


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


@pytest.mark.parametrize("op", [C.SOFTMAX, C.LAYERNORM, C.RMSNORM, C.QUANT_INT8])
@pytest.mark.parametrize("dt", [C.F32, C.BF16, C.FP8_E4M3])
def test_reduction_reuse_ops_are_candidates(op, dt):
    d = C.dataflow(op, dt)
    assert d.stages == 1 and d.b_reread == {C.F32: 4, C.BF16: 2, C.FP8_E4M3: 1}[dt]
    for P in (1, 2, 4, 8, 16):
        assert C.screen(d, P) == (C.SCREEN_CANDIDATE, 2)  # K = 2L, independent of P


@pytest.mark.parametrize("op,verdict", [(C.LOGSUMEXP, C.SCREEN_NO_REUSE), (C.STENCIL, C.SCREEN_NO_REUSE),
                                        (C.SCAN, C.SCREEN_ORDERED), (C.SELECT, C.SCREEN_REMOTE_STATE)])
def test_negative_controls_are_rejected(op, verdict):
    d = C.dataflow(op)
    for P in (2, 4, 8, 16):
        v, K = C.screen(d, P)
        assert v == verdict
        if op == C.SCAN:
            assert K == 2 * (P - 1)  # one dependent carry exchange per CTA boundary


def test_plan_of_a_control_is_the_global_path():
    for op, verdict in ((C.SCAN, C.SCREEN_ORDERED), (C.STENCIL, C.SCREEN_NO_REUSE)):
        p, v = C.plan_control(op, 4096, 262144)
        assert v == verdict and p.path == C.PATH_TWO_PASS and p.cluster_size == 1 and p.source == 3


def test_screen_and_control_arguments_are_checked():
    with pytest.raises(C.CreditError):
        C.dataflow(99)
    with pytest.raises(C.CreditError):
        C.screen(C.dataflow(C.SOFTMAX), 17)
    with pytest.raises(C.CreditError):
        C.plan_control(C.SOFTMAX, 4, 16)
    # argument checks run before anything touches a GPU (stream 0: no torch stream needed)
    assert C.run_control_status(C.SCAN, None, None, rows=4, cols=16, stream=0) == C.ERR_INVALID_ARG
    assert C.run_control_status(C.SOFTMAX, None, None, rows=4, cols=16, stream=0) == C.ERR_INVALID_ARG
