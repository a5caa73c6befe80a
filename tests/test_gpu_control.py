"""GPU parity of the negative-control ops (row scan and row stencil, which
the screen of Sec. III-D rejects for the cluster path and runs on the
non-DSMEM global path) against the FP64 oracle: rows with ragged tails,
unaligned rows and strides, in-place scans, several stencil radii.

Bounds: a scan output is a sum of up to N FP32 terms, so |y - y*| <= 1e-5 of
the sum of the magnitudes of its terms (sum_{j <= i} |x_j|); a stencil output
within 1e-5 of sum_k |w_k x_{i+k}|."""
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


def check_scan(x64, y):
    ref = O.scan(x64)
    bound = 1e-5 * np.cumsum(np.abs(x64), axis=1) + 1e-30
    e = np.abs(y - ref) / bound
    assert np.all(np.isfinite(e)) and e.max() <= 1.0, e.max()


@pytest.mark.parametrize("cols", [1, 7, 2048, 4099, 65536, 262147])
def test_scan_matches_oracle(cols):
    x = synth.outliers(37, cols, seed=cols)
    out = torch.full((37, cols), float("nan"), device="cuda")
    C.run_control(C.SCAN, x.cuda(), out)
    torch.cuda.synchronize()
    check_scan(x.double().numpy(), out.double().cpu().numpy())


def test_scan_unaligned_strided_and_in_place():
    cols, ld = 5001, 5003
    x = synth.normal(19, ld, seed=3) + 10.0  # a growing sum
    base = torch.zeros(19 * ld + 1, device="cuda")
    base[1:] = x.reshape(-1).cuda()
    out = torch.full((19, cols + 2), float("nan"), device="cuda")
    C.run_control(C.SCAN, base[1:], out, rows=19, cols=cols, ld_in=ld, ld_out=cols + 2)
    torch.cuda.synchronize()
    check_scan(x[:, :cols].double().numpy(), out[:, :cols].double().cpu().numpy())
    assert torch.isnan(out[:, cols:]).all()
    xi = x.cuda()
    C.run_control(C.SCAN, xi, xi)  # in place
    torch.cuda.synchronize()
    check_scan(x.double().numpy(), xi.double().cpu().numpy())


@pytest.mark.parametrize("w", [[0.25, 0.5, 0.25], [0.1, -0.2, 0.4, -0.2, 0.1], [1.0], list(np.linspace(-1, 1, 17))])
@pytest.mark.parametrize("cols", [3, 1000, 65541])
def test_stencil_matches_oracle(w, cols):
    x = synth.outliers(11, cols, seed=len(w) + cols)
    wt = torch.tensor(w, dtype=torch.float32)
    out = torch.full((11, cols), float("nan"), device="cuda")
    C.run_control(C.STENCIL, x.cuda(), out, weights=wt.cuda())
    torch.cuda.synchronize()
    x64, w64 = x.double().numpy(), wt.double().numpy()
    ref = O.stencil(x64, w64)
    mag = O.stencil(np.abs(x64), np.abs(w64))
    e = np.abs(out.double().cpu().numpy() - ref) / (1e-5 * mag + 1e-30)
    assert np.all(np.isfinite(e)) and e.max() <= 1.0


def test_control_refusals_launch_nothing():
    x = torch.zeros(4, 64, device="cuda")
    w = torch.ones(3, device="cuda")
    n0 = C.launch_count()
    assert C.run_control_status(C.STENCIL, x, x, weights=w) == C.ERR_INVALID_ARG            # in place
    assert C.run_control_status(C.STENCIL, x, torch.empty_like(x)) == C.ERR_INVALID_ARG      # no weights
    assert C.run_control_status(C.STENCIL, x, torch.empty_like(x), weights=torch.ones(19, device="cuda")) == \
        C.ERR_INVALID_ARG                                                                    # radius 9
    assert C.launch_count() == n0
