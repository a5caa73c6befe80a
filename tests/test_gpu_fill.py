"""GPU tests of cluster plans with a fill: the last rows of the call run on the
split two-pass path, on a library stream forked from and joined back into the
caller's stream, over the SMs the clusters leave idle.

Checks: oracle parity for every op, both retention tiers and both cluster
sizes that leave SMs idle; bit equality with a pure cluster run on the first
rows and a pure two-pass run on the last rows (rows are independent, the
kernels the same); CUDA-graph capture of the fork / join; the refusals; and
the occupancy query the planner uses.
"""
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


def affine(op, cols):
    from paper_2609_01864_gb300 import synth
    if op in (C.LAYERNORM, C.RMSNORM):
        g, b = synth.gamma_beta(cols, seed=5)
        return g, (b if op == C.LAYERNORM else None)
    return None, None


def fill_split(cols, isz):
    return max(1, min(8, cols * isz // (512 << 10)))


@pytest.mark.parametrize("share", [0.15, 0.4])
@pytest.mark.parametrize("retain", [C.RETAIN_SMEM, C.RETAIN_TMEM])
@pytest.mark.parametrize("P", [8, 16])
@pytest.mark.parametrize("op", [C.SOFTMAX, C.LOGSUMEXP, C.LAYERNORM, C.RMSNORM])
def test_fill_matches_oracle(op, P, retain, share):
    if op == C.LOGSUMEXP and retain == C.RETAIN_TMEM:
        pytest.skip("logsumexp has no tensor-memory form")
    rows, cols = 90, 70001
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers" if op in (C.LAYERNORM, C.RMSNORM) else "normal",
                        std=3.0, seed=P + retain + int(100 * share))
    g, b = affine(op, cols)
    plan = C.make_plan(C.PATH_CLUSTER, P, retain=retain, fill_share=share)
    U.check_against_oracle(op, x, None, plan=plan, gamma=g, beta=b)


@pytest.mark.parametrize("dt", [(C.BF16, C.BF16), (C.FP8_E4M3, C.F32), (C.F32, C.FP8_E4M3)],
                         ids=lambda d: f"{d[0]}to{d[1]}")
@pytest.mark.parametrize("op", [C.SOFTMAX, C.RMSNORM])
def test_fill_low_precision(op, dt):
    tin, tout = dt
    x, s = U.make_input(tin, 70, 131072, std=3.0, seed=tin * 3 + tout)
    g, b = affine(op, 131072)
    plan = C.make_plan(C.PATH_CLUSTER, 16, fill_share=0.3)
    U.check_against_oracle(op, x, s, out_dtype=tout, plan=plan, gamma=g, beta=b)


@pytest.mark.parametrize("op", [C.SOFTMAX, C.LAYERNORM, C.RMSNORM])
def test_fill_rows_are_bitwise_the_two_paths(op):
    rows, cols, P, share = 200, 262144, 8, 0.3
    x, _ = U.make_input(C.F32, rows, cols, kind="outliers", std=2.0, seed=31)
    g, b = affine(op, cols)
    n_fill = int(rows * share + 0.5)
    both, _ = U.run_gpu(op, x, None, plan=C.make_plan(C.PATH_CLUSTER, P, retain=C.RETAIN_TMEM, fill_share=share),
                        gamma=g, beta=b)
    cl, _ = U.run_gpu(op, x[: rows - n_fill], None, plan=C.make_plan(C.PATH_CLUSTER, P, retain=C.RETAIN_TMEM),
                      gamma=g, beta=b)
    tp, _ = U.run_gpu(op, x[rows - n_fill:], None,
                      plan=C.make_plan(C.PATH_TWO_PASS, ctas_per_row=fill_split(cols, 4)), gamma=g, beta=b)
    torch.cuda.synchronize()
    assert torch.equal(both[: rows - n_fill], cl)
    assert torch.equal(both[rows - n_fill:], tp)


def test_fill_in_a_cuda_graph():
    rows, cols = 128, 131072
    x = torch.randn(rows, cols, device="cuda")
    y_eager = torch.empty_like(x)
    y_graph = torch.zeros_like(x)
    plan = C.make_plan(C.PATH_CLUSTER, 16, retain=C.RETAIN_TMEM, fill_share=0.3)
    C.run_ex(C.SOFTMAX, x, y_eager, plan=plan)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        C.run_ex(C.SOFTMAX, x, y_graph, plan=plan)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    y_graph.zero_()
    with torch.cuda.graph(graph):
        C.run_ex(C.SOFTMAX, x, y_graph, plan=plan)
    graph.replay()
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    assert torch.equal(y_graph, y_eager)


def test_fill_refusals_launch_nothing():
    x = torch.randn(64, 65536, device="cuda")
    y = torch.empty_like(x)
    n0 = C.launch_count()
    bad = [C.make_plan(C.PATH_TWO_PASS, ctas_per_row=2, fill_share=0.2),  # fill only for cluster plans
           C.make_plan(C.PATH_ONE_CTA, fill_share=0.2),
           C.make_plan(C.PATH_CLUSTER, 8, fill_share=0.95),                  # above the 0.9 limit
           C.make_plan(C.PATH_CLUSTER, 8, fill_share=-0.1),
           C.make_plan(C.PATH_CLUSTER, 8, fill_share=float("nan")),
           C.make_plan(C.PATH_CLUSTER, 8, fill_share=0.2, fill_g=5000)]
    for p in bad:
        assert C.run_ex_status(C.RMSNORM, x, y, plan=p) == C.ERR_UNSUPPORTED
    assert C.launch_count() == n0


def test_max_clusters_query():
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    x = torch.randn(64, 262144, device="cuda")
    y = torch.empty_like(x)
    for P in (2, 4, 8, 16):
        n = C.max_clusters(C.RMSNORM, x, y, C.make_plan(C.PATH_CLUSTER, P, retain=C.RETAIN_TMEM))
        if P >= 8:
            assert 0 < n and n * P <= sm
    assert C.max_clusters(C.RMSNORM, x, y, C.make_plan(C.PATH_TWO_PASS, ctas_per_row=2)) == 0
    assert C.max_clusters(C.RMSNORM, x, y, C.make_plan(C.PATH_CLUSTER, 2, retain=C.RETAIN_TMEM)) == 0  # 512 KiB slice
