"""CPU tests of host logic around the kernels: the planner's feature vector,
the sweep's timing files, and the bench's kernel naming and profitability
pairs.  Nothing here needs a GPU."""
import math
import os
import sys

import numpy as np
import pytest

from paper_2609_01864_gb300 import build as B
from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import sweep as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    C.lib()


def test_features_of_a_cluster_candidate():
    f = C.mlp_features(C.RMSNORM, C.BF16, C.BF16, 4096, 131072, C.PATH_CLUSTER, 8, 1, C.RETAIN_TMEM, 0.25)
    assert f.shape == (C.MLP_FEATURES,) == (21,)
    assert f[0] == 12 and f[1] == 17
    assert list(f[2:5]) == [0, 1, 0]            # input BF16
    assert list(f[5:9]) == [0, 0, 0, 1]         # RMSNorm
    assert list(f[9:12]) == [0, 0, 1]           # cluster path
    assert f[12] == 3 and f[13] == 0            # log2 P, log2 G
    assert f[14] == pytest.approx(math.log2(4096 * 131072 * 4))
    assert f[15] == 2                           # output bytes per element
    assert f[16] == pytest.approx(math.log2(131072 * 2 / 8 + 1))
    assert f[17] == pytest.approx(math.log2(4096 * 8 / 152))
    assert f[18] == 1 and f[19] == pytest.approx(0.25)
    assert f[20] == 1                           # 131072 BF16 = 16 K groups: every row on the 16-byte grid


def test_features_ignore_retention_and_fill_where_they_do_not_apply():
    tp = C.mlp_features(C.SOFTMAX, C.F32, C.F32, 64, 65536, C.PATH_TWO_PASS, 1, 4, C.RETAIN_TMEM, 0.3)
    assert tp[18] == 0 and tp[19] == 0 and tp[13] == 2
    one = C.mlp_features(C.LAYERNORM, C.F32, C.F32, 64, 8192, C.PATH_ONE_CTA, 1, 1, C.RETAIN_TMEM, 0.3)
    assert one[18] == 1 and one[19] == 0
    lse = C.mlp_features(C.LOGSUMEXP, C.FP8_E4M3, C.BF16, 10, 1000, C.PATH_ONE_CTA, 1, 1)
    assert lse[15] == 0                         # one FP32 value per row, counted in the bytes instead
    assert lse[14] == pytest.approx(math.log2(10 * 1000 * 1 + 10 * 4))
    assert lse[20] == 0                         # 1000 FP8 codes: rows off the 16-byte grid
    assert C.mlp_features(C.SOFTMAX, C.F32, C.F32, 8, 1002, C.PATH_TWO_PASS, 1, 1)[20] == 0
    assert C.mlp_features(C.SOFTMAX, C.BF16, C.BF16, 8, 1000, C.PATH_TWO_PASS, 1, 1)[20] == 1


@pytest.mark.parametrize("bad", [dict(op=4), dict(rows=0), dict(path=3), dict(retain=3), dict(fill_share=1.5),
                                 dict(fill_share=float("nan"))])
def test_features_reject_bad_arguments(bad):
    a = dict(op=C.SOFTMAX, in_dtype=C.F32, out_dtype=C.F32, rows=8, cols=64, path=C.PATH_CLUSTER, P=2, G=1,
             retain=0, fill_share=0.0)
    a.update(bad)
    with pytest.raises(C.CreditError):
        C.mlp_features(**a)


def test_sweep_timings_round_trip_and_older_forms(tmp_path):
    rows = [dict(shape=0, op=3, dtype=0, rows=512, cols=524288, path=C.PATH_CLUSTER, P=16, G=1, retain=2,
                 fill=0.15, us=2708.125),
            dict(shape=1, op=0, dtype=1, rows=7, cols=100, path=C.PATH_TWO_PASS, P=1, G=4, retain=0, fill=0.0,
                 us=5.5)]
    p = tmp_path / "t.csv"
    S.write_csv(str(p), rows)
    assert S.read_csv(str(p)) == rows
    old9 = tmp_path / "old9.csv"
    old9.write_text("shape,op,dtype,rows,cols,path,P,G,us\n0,0,2,81,7473,0,1,1,22.432\n3,1,0,9,99,1,1,2,4.0\n")
    r9 = S.read_csv(str(old9))
    assert (r9[0]["retain"], r9[0]["fill"]) == (C.RETAIN_SMEM, 0.0)   # one-CTA staged in shared memory
    assert (r9[1]["retain"], r9[1]["G"]) == (C.RETAIN_AUTO, 2)        # two-pass: no retention
    old10 = tmp_path / "old10.csv"
    old10.write_text("shape,op,dtype,rows,cols,path,P,G,retain,us\n5,2,0,64,65536,2,4,1,2,80.5\n")
    r10 = S.read_csv(str(old10))[0]
    assert (r10["retain"], r10["fill"], r10["us"]) == (2, 0.0, 80.5)
    bad = tmp_path / "bad.csv"
    bad.write_text("h\n1,2,3\n")
    with pytest.raises(ValueError):
        S.read_csv(str(bad))


def test_shipped_timings_parse():
    rows = S.read_csv(os.path.join(ROOT, "paper_2609_01864_gb300", "data", "sweep_gb300.csv"))
    assert len(rows) > 1000
    assert all(r["us"] > 0 and 0.0 <= r["fill"] <= 0.9 for r in rows)
    assert {r["path"] for r in rows} == {C.PATH_ONE_CTA, C.PATH_TWO_PASS, C.PATH_CLUSTER}


def test_kernel_names(monkeypatch):
    monkeypatch.delenv("CREDIT_RETAIN", raising=False)
    mk = C.make_plan
    assert bench.kernel_name(mk(C.PATH_TWO_PASS, ctas_per_row=1), C) == "k_tp_fused"
    assert bench.kernel_name(mk(C.PATH_TWO_PASS, ctas_per_row=4), C) == "k_tp_split"
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 16, retain=C.RETAIN_TMEM, fill_share=0.4), C) == "k_ring_tm+fill"
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 8, retain=C.RETAIN_SMEM, fill_share=0.2), C) == "k_ring+fill"
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 4, retain=C.RETAIN_SMEM), C, 65536) == "k_ring"
    # AUTO: tensor memory for slices above 32 KiB that fit 8 chunks of 16 KiB
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 4, retain=C.RETAIN_AUTO), C, 65536) == "k_ring_tm"
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 8, retain=C.RETAIN_AUTO), C, 65536) == "k_ring"      # 32 KiB
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 2, retain=C.RETAIN_AUTO), C, 131072) == "k_ring"     # 256 KiB
    monkeypatch.setenv("CREDIT_RETAIN", "smem")
    assert bench.kernel_name(mk(C.PATH_CLUSTER, 4, retain=C.RETAIN_AUTO), C, 65536) == "k_ring"


def test_profitability_pairs():
    rows = [dict(op="layernorm", cols=16384, analytic_cluster=False, measured_cluster=False),
            dict(op="layernorm", cols=65536, analytic_cluster=True, measured_cluster=False),
            dict(op="layernorm", cols=131072, analytic_cluster=True, measured_cluster=True),
            dict(op="rmsnorm", cols=131072, analytic_cluster=False, measured_cluster=True),
            dict(op="rmsnorm", cols=65536, analytic_cluster=False, measured_cluster=False)]
    p = bench.profitability(rows)
    assert p["pairs"] == 5 and p["sign_agreement"] == 3
    assert p["n_star"] == {"layernorm": {"analytic": 65536, "measured": 131072},
                           "rmsnorm": {"analytic": None, "measured": 131072}}


def test_algorithmic_bytes_count_one_read_and_one_write():
    assert bench.algorithmic_bytes(4096, 524288, C.LAYERNORM) == 4096 * 524288 * 4 * 2


def test_traffic_record_is_used_only_for_the_kernel_source_it_was_taken_on(tmp_path, monkeypatch):
    """profiles/traffic.json is keyed by a hash of the row-kernel sources: the bench reports a record's DRAM bytes
    as roofline.traffic only while the hash matches the sources as they are, and null after any kernel edit."""
    import json
    recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))["records"]
    assert recs
    for r in recs:
        assert r["dram_bytes"] == r["dram_read"] + r["dram_write"]
        assert 0.9 < r["dram_bytes"] / r["algorithmic_bytes"] < 1.6
    r = dict(recs[0])
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda: "current-sources")
    r["source_sha"] = "current-sources"
    (prof / "traffic.json").write_text(json.dumps({"records": [r]}))
    assert bench.traffic_record(r["kernel"], r["op"], r["cols"]) == r
    assert bench.traffic_record(r["kernel"], r["op"], r["cols"] + 1) is None
    r["source_sha"] = "older-sources"
    (prof / "traffic.json").write_text(json.dumps({"records": [r]}))
    assert bench.traffic_record(r["kernel"], r["op"], r["cols"]) is None


def test_sweep_shape_width_modes():
    """The training-only wide-corner shapes cycle through drawn widths, the nearest power of two and widths
    rounded down to a multiple of 16; the draw itself (op, dtype, rows) is unchanged by the mode."""
    from paper_2609_01864_gb300 import synth
    kw = dict(seed=17, rows_log2=(10.0, 14.0), cols_log2=(14.0, 20.0))
    plain = synth.sweep_shapes(90, **kw)
    moded = synth.sweep_shapes(90, col_modes=("any", "pow2", "align16"), **kw)
    for i, (a, b) in enumerate(zip(plain, moded)):
        assert a[:3] == b[:3]
        cols = b[3]
        if i % 3 == 0:
            assert cols == a[3]
        elif i % 3 == 1:
            assert cols & (cols - 1) == 0 and a[3] / 2 <= cols <= 2 * a[3]
        else:
            assert cols % 16 == 0 and a[3] - 16 < cols <= a[3]
    assert synth.sweep_shapes(50) == synth.sweep_shapes(50, col_modes=("any",))


def test_sweep_reuses_only_identical_shapes():
    """--reuse-csv keeps an earlier sweep's timings for a shape id only where every recorded row matches the
    shape now drawn at that id, and times the rest (including ids the earlier sweep never had)."""
    def row(i, op, dt, r, c, us):
        return dict(shape=i, op=op, dtype=dt, rows=r, cols=c, path=1, P=1, G=1, retain=0, fill=0.0, us=us)
    old = [row(0, 0, 0, 64, 1024, 1.0), row(0, 0, 0, 64, 1024, 2.0), row(1, 2, 1, 128, 4096, 3.0),
           row(2, 3, 2, 256, 8192, 4.0)]
    shapes = [(0, 0, 64, 1024), (2, 1, 128, 4000), (3, 2, 256, 8192), (1, 0, 512, 2048)]
    kept, todo = S.reusable_timings(old, shapes)
    assert [r["us"] for r in kept] == [1.0, 2.0, 4.0]
    assert todo == [1, 3]


def test_learned_pick_prefers_a_plan_without_fill_only_within_the_tie_margin():
    """The learned planner's choice as the sweep scores it: the lowest prediction, except that within
    FILL_TIE_LOG2 of it the lowest prediction without a fill wins (two-pass and one-CTA plans count as
    plans without a fill); ties at equal predictions keep the first candidate."""
    def cand(name, pred, fill=0.0):
        return dict(name=name, pred_log2us=pred, fill=fill)
    eps = S.FILL_TIE_LOG2
    # a fill ahead by less than the margin: the plain cluster plan
    c = [cand("c16_f0.15", 1.000, 0.15), cand("c16", 1.000 + 0.4 * eps), cand("tp4", 1.5)]
    assert S.learned_pick(c)["name"] == "c16"
    # a fill ahead by more than the margin: the fill
    c = [cand("c16_f0.15", 1.000, 0.15), cand("c16", 1.000 + 2.0 * eps), cand("tp4", 1.5)]
    assert S.learned_pick(c)["name"] == "c16_f0.15"
    # only fills near the minimum: the lowest of them
    c = [cand("c8_f0.2", 2.0, 0.2), cand("c8_f0.15", 1.99, 0.15), cand("tp1", 3.0)]
    assert S.learned_pick(c)["name"] == "c8_f0.15"
    # among plans without a fill inside the margin, the lowest; equal predictions keep the first
    c = [cand("c4", 1.004), cand("c2", 1.002), cand("c2b", 1.002), cand("c8_f0.3", 1.0, 0.3)]
    assert S.learned_pick(c)["name"] == "c2"
