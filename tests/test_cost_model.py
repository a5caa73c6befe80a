"""The analytic profitability model (Sec. III-D): oracle pins and the
library's implementation against the oracle (CPU only).

Pins are values worked out by hand from the equations on fabricated inputs
(the arithmetic is written next to each), plus structural facts the paper
states: scalar-output reductions (b_reread = 0) are never profitable, the
saved time grows with the row width, the P sources' remote stores are not
multiplied by P, and Eq. 6 gives 1920 remote bytes per row at P = 16, q = 2.
"""
import math
import random

import pytest

import oracle.cost_model as CM

BASE = dict(M=4096, N=65536, P=4, T_B_us=600.0, T_ctrl_us=10.0, b_B=12.0, b_reread=4.0, b_keep=4.0, b_in=4.0,
            s_bytes=4.0, q_sum=2.0, active_clusters=38, f_mhz=1900.0, B_smem_read=128.0, B_smem_store=128.0,
            B_dsm_store=20.0, B_peak_gbs=6800.0)


def test_worked_example_by_hand():
    t = CM.evaluate(BASE)
    # W = ceil(4096 / 38) = 108
    assert t["W"] == 108
    # B_eff = 4096 * 65536 * 12 B / 600 us = 3221225472 / 600 B/us = 5368.70912 GB/s
    assert t["B_eff_gbs"] == pytest.approx(5368.70912, rel=1e-12)
    # T_save = 600 * 4 / 12 = 200 us
    assert t["T_save_us"] == pytest.approx(200.0, rel=1e-15)
    # T_replay = 108 * 16384 * 4 / (1900 * 128) = 7077888 / 243200 = 29.1031578947 us
    assert t["T_replay_us"] == pytest.approx(7077888 / 243200, rel=1e-15)
    # T_DSM = 4 * 108 * 3 * 2 / (1900 * 20) = 2592 / 38000 us
    assert t["T_dsm_us"] == pytest.approx(2592 / 38000, rel=1e-15)
    # T_SMEM^w equals T_replay here (same rate); T_input = M N b_in / B_eff = 200 us > it, so no deposit
    assert t["T_input_us"] == pytest.approx(200.0, rel=1e-12)
    assert t["T_deposit_us"] == 0.0
    # dT = 200 - 10 - 29.1031578947 - 0 - 0.0682105263
    assert t["dT_us"] == pytest.approx(200 - 10 - 7077888 / 243200 - 2592 / 38000, rel=1e-13)


def test_ablation_uses_peak_and_serial_staging():
    t = CM.evaluate(BASE, ablation=True)
    # T_save = M N b_reread / B_peak = 268435456 * 4 / 6.8e6 B/us = 157.903209... us
    assert t["T_save_us"] == pytest.approx(268435456 * 4 / 6.8e6, rel=1e-15)
    assert t["T_deposit_us"] == pytest.approx(t["T_smem_w_us"], rel=1e-15)


def test_no_reread_is_never_profitable():
    for P in (2, 4, 8, 16):
        t = CM.evaluate(dict(BASE, P=P, b_reread=0.0, b_B=4.0))  # log-sum-exp: one pass, scalar output
        assert t["T_save_us"] == 0.0 and t["dT_us"] < 0
    assert CM.pick({2: -1.0, 4: -0.5}) is None
    assert CM.pick({2: 3.0, 4: 5.0, 8: -1.0}) == 4


def test_saved_time_grows_with_width_at_fixed_rate():
    last = -1e30
    for N in (4096, 16384, 65536, 262144):
        T_B = N * 4096 * 12 / 5.0e6  # a baseline that streams at 5 TB/s
        t = CM.evaluate(dict(BASE, N=N, T_B_us=T_B, T_ctrl_us=0.0))
        assert t["T_save_us"] > last
        last = t["T_save_us"]


def test_remote_store_time_not_multiplied_by_P():
    t4 = CM.evaluate(dict(BASE, P=4))
    t8 = CM.evaluate(dict(BASE, P=8))
    # (P - 1) scaling only: 7/3 at equal W
    assert t8["T_dsm_us"] / t4["T_dsm_us"] == pytest.approx(7 / 3, rel=1e-12)


def test_capacity_and_protocol_equations():
    S_max = 232448  # GB300 opt-in shared memory per block
    # FP32 64K row (256 KiB): illegal on one CTA, legal on two (Eq. 3 capacity)
    assert not CM.capacity_ok(65536, 1, 4, 2304, S_max)
    assert CM.capacity_ok(65536, 2, 4, 2304, S_max)
    # FP32 512K row needs P = 16
    assert not CM.capacity_ok(524288, 8, 4, 2304, S_max) and CM.capacity_ok(524288, 16, 4, 2304, S_max)
    assert CM.dsmem_protocol(4, 16, [2]) == (1920, 0.0, 2)
    assert CM.hbm_traffic(4 * 65536, 65536, 4) == (8 * 65536, 4 * 65536)
    assert CM.crossover([4096, 8192, 16384], {4096: {2: -1.0}, 8192: {2: -0.1, 4: 0.2}, 16384: {2: 1.0}}) == 8192


def test_library_model_matches_oracle():
    from paper_2609_01864_gb300 import build as B
    from paper_2609_01864_gb300 import credit as C
    B.build()
    rng = random.Random(5)
    for _ in range(500):
        inp = dict(M=rng.choice([64, 300, 4096, 65536]), N=rng.choice([1000, 4096, 65536, 1 << 20]),
                   P=rng.choice([2, 4, 8, 16]), T_B_us=rng.uniform(5, 5000), T_ctrl_us=rng.uniform(0, 50),
                   b_B=rng.choice([2.0, 4.0, 8.0, 12.0]), b_reread=rng.choice([0.0, 1.0, 2.0, 4.0]),
                   b_keep=rng.choice([1.0, 2.0, 4.0]), b_in=rng.choice([1.0, 2.0, 4.0]), s_bytes=4.0,
                   q_sum=rng.choice([1.0, 2.0, 3.0]), active_clusters=rng.choice([7, 15, 38, 152]),
                   f_mhz=rng.uniform(1200, 2100), B_smem_read=rng.uniform(32, 128),
                   B_smem_store=rng.uniform(32, 128), B_dsm_store=rng.uniform(1, 40),
                   B_peak_gbs=rng.uniform(3000, 8000))
        for abl in (False, True):
            ref = CM.evaluate(inp, ablation=abl)
            got = C.model_eval(**inp, ablation=int(abl))
            for k, v in ref.items():
                assert got[k] == pytest.approx(v, rel=1e-12, abs=1e-9), (k, inp, abl)
