"""The bounded-wait error path on the GPU, without a fault: a one-CTA call on
one row of one chunk whose first chunk barrier expects 16 bytes more than its
bulk copy delivers (credit_set_wait_test) makes the reducers' wait run out
after 1 ms.  The call returns, credit_device_error() reports
CREDIT_ERR_TIMEOUT once (the word is cleared by the read), and the next
normal calls are parity-green.  Nothing is left in flight: the one copy that
is issued completes, and the barrier is never reused."""
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
    C.set_wait_test(0, 0)


def test_bounded_wait_gives_up_and_reports_timeout():
    plan = C.make_plan(C.PATH_ONE_CTA, retain=C.RETAIN_SMEM)
    x = torch.randn(1, 1024, device="cuda")
    y = torch.empty_like(x)
    assert C.device_error() == C.OK
    C.set_wait_test(1_000_000, 16)
    try:
        C.run_ex(C.SOFTMAX, x, y, plan=plan)
        torch.cuda.synchronize()
        assert C.device_error() == C.ERR_TIMEOUT
        assert C.device_error() == C.OK  # read and cleared
        # the knob is refused, launching nothing, wherever the barrier would be reused
        x2 = torch.randn(2, 1024, device="cuda")
        n0 = C.launch_count()
        assert C.run_ex_status(C.SOFTMAX, x2, torch.empty_like(x2), plan=plan) == C.ERR_UNSUPPORTED
        assert C.run_ex_status(C.SOFTMAX, x, y, plan=C.make_plan(C.PATH_CLUSTER, 2)) == C.ERR_UNSUPPORTED
        assert C.launch_count() == n0
    finally:
        C.set_wait_test(0, 0)
    # the context stays usable: normal calls afterwards match the oracle
    xs = torch.randn(64, 20000) * 3
    for p in (plan, C.make_plan(C.PATH_CLUSTER, 4), None):
        U.check_against_oracle(C.SOFTMAX, xs, None, plan=p)
    assert C.device_error() == C.OK


def test_wait_test_arguments_are_checked():
    for bad in ((-1, 0), (0, -16), (0, 8), (0, 1 << 21)):
        with pytest.raises(C.CreditError):
            C.set_wait_test(*bad)
