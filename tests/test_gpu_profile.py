"""GPU checks of the profiling layer (Sec. III-A microbenchmarks, the
control kernel of Sec. III-D) and of planning from a calibration."""
import os

import pytest
import torch

from paper_2609_01864_gb300 import credit as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield


def test_microbenchmarks_are_sane():
    m = C.microbench(runs=5)
    assert m["distinct_sms"] == 1                       # the two CTAs ran on different SMs
    assert 5 < m["lat_local_cycles"] < m["lat_remote_cycles"] < 5000
    assert m["rate_local_read"] > m["rate_remote_read"] > 0
    assert all(v > 0 for v in m["rate_remote_store"])
    assert all(v > 0 for v in m["sync_cycles"])
    assert 500 < m["sm_clock_mhz"] < 2500


def test_control_kernel_times_and_excess():
    t1 = C.control_time(C.SOFTMAX, 4096, 4096, C.F32, 1, reps=5)
    t16 = C.control_time(C.SOFTMAX, 4096, 65536, C.F32, 16, reps=5)
    assert t1 > 0 and t16 > 0
    assert C.device_error() == C.OK


def test_calibrate_load_and_plan(tmp_path, monkeypatch):
    monkeypatch.setenv("CREDIT_MODEL", "analytic")
    path = str(tmp_path / "gb300.calib")
    C.calibrate(path, max_bytes=1 << 28)
    text = open(path).read()
    assert text.startswith("credit-calibration 1") and "\ntb " in text and "\ntctrl " in text
    C.load_model(path)
    p = C.plan(C.RMSNORM, 4096, 65536, C.F32)
    assert p.source == 0 and p.predicted_us > 0
    p = C.plan(C.LOGSUMEXP, 4096, 262144, C.F32)
    assert p.path == C.PATH_TWO_PASS                     # b_reread = 0: never the cluster path
    x = torch.randn(256, 8192, device="cuda")
    y = torch.empty_like(x)
    C.run_ex(C.SOFTMAX, x, y)                           # the planner's plan runs
    torch.cuda.synchronize()
    assert torch.allclose(y.sum(dim=1), torch.ones(256, device="cuda"), atol=1e-4)


def test_committed_calibration_and_learned_planner(monkeypatch):
    data = os.path.join(os.path.dirname(C.__file__), "data", "gb300.calib")
    monkeypatch.delenv("CREDIT_MODEL", raising=False)
    C.load_model(data)                                    # loads the MLP weights it names
    p = C.plan(C.LAYERNORM, 4096, 65536, C.F32)
    assert p.source == 1 and p.predicted_us > 0           # learned model by default
    for cols in (16384, 262144, 1 << 20):
        q = C.plan(C.LOGSUMEXP, 4096, cols, C.F32)
        assert q.path != C.PATH_CLUSTER                   # the analytic screen's veto (no reread to save)
    monkeypatch.setenv("CREDIT_MODEL", "analytic")
    assert C.plan(C.LAYERNORM, 4096, 65536, C.F32).source == 0
