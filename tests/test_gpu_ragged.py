"""Ragged batches (rows of uneven width, mixed softmax / RMSNorm, packed with
no alignment padding) through one persistent graph-captured launch, against
the FP64 oracle row by row."""
import os

import numpy as np
import pytest
import torch

from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

import parity_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _init():
    from paper_2609_01864_gb300 import build as B
    B.build()
    C.init()
    yield


def packed_batch(widths, ops, dtype, seed=0):
    offs = np.concatenate([[0], np.cumsum(widths)[:-1]]).astype(np.int64)
    total = int(np.sum(widths))
    g = torch.Generator().manual_seed(seed)
    flat = (torch.randn(total, generator=g) * 2.0)
    flat = flat.to(C.TORCH_DTYPE[dtype])
    rows = [(int(o), int(o), int(w), int(op)) for o, w, op in zip(offs, widths, ops)]
    return flat, rows, offs


def check_rows(flat_in, flat_out_dev, rows, dtype, pick):
    out = flat_out_dev.cpu()
    for i in pick:
        io, oo, w, op = rows[i]
        x = flat_in[io:io + w].reshape(1, w)
        ref = U.reference(op, dtype, x)
        y = U.to64(out[oo:oo + w].reshape(1, w))
        assert U.error_metric(op, dtype, y, ref) <= 1.0, (i, w, op)


@pytest.mark.parametrize("force", [("16", "13", "256"), ("4", "2", "128"), ("8", "6", "256")],
                         ids=["wide", "huge", "mixed"])
def test_ragged_kinds_match_oracle(force, monkeypatch):
    monkeypatch.setenv("CREDIT_RAGGED_P", force[0])
    monkeypatch.setenv("CREDIT_RAGGED_CHUNKS", force[1])
    monkeypatch.setenv("CREDIT_RAGGED_THREADS", force[2])
    widths, ops = synth.ragged_widths(120, seed=11)
    widths = widths.numpy()
    ops = ops.numpy()
    widths[:3] = [1, 7, 1048576]  # tiny and maximal rows
    for dt in (C.BF16, C.F32):
        flat, rows, _ = packed_batch(widths, ops, dt, seed=dt)
        d_in = flat.cuda()
        d_out = torch.full_like(d_in, float("nan"))
        R = C.Ragged(rows, dt, d_in, d_out, tune=False)
        info = R.info()
        R.run()
        torch.cuda.synchronize()
        assert C.device_error() == C.OK
        check_rows(flat, d_out, rows, dt, range(len(rows)))
        R.close()
        assert info["items"] == info["narrow_items"] + info["wide_items"] + info["huge_items"]


@pytest.mark.parametrize("force", [("16", "2", "256", "1"), ("2", "1", "128", "2"), ("8", "13", "256", "1"),
                                   ("8", "3", "256", "2")],
                         ids=["p16_small_cap", "p2_vw2", "p8", "p8_vw2"])
def test_ragged_every_width_class(force, monkeypatch):
    """Rows sized so that every sub-cluster width w = 1, 2, 4, ..., P occurs, in runs whose lengths are
    not multiples of P / w (items with idle sub-groups), next to rows that stream (huge); both vector
    widths."""
    monkeypatch.setenv("CREDIT_RAGGED_P", force[0])
    monkeypatch.setenv("CREDIT_RAGGED_CHUNKS", force[1])
    monkeypatch.setenv("CREDIT_RAGGED_THREADS", force[2])
    monkeypatch.setenv("CREDIT_RAGGED_VW", force[3])
    P, cap = int(force[0]), int(force[1]) * 16384
    rng = np.random.default_rng(int(force[0]) * 7 + int(force[1]))
    for dt in (C.BF16, C.F32):
        isz = 2 if dt == C.BF16 else 4
        widths = []
        w = 1
        while w <= P:  # per class w: more elements than w / 2 CTAs can stage, few enough for w
            lo = (cap - 32) * (w // 2) // isz + 8 if w > 1 else 1
            hi = (cap - 48) * w // isz - 16 * w
            n = int(rng.integers(1, 2 * (P // w) + 2))
            widths += list(rng.integers(lo, hi, n))
            w *= 2
        widths += [cap * P // isz + 1000, cap * P // isz + 12345]  # beyond the cluster's staging: huge
        widths += [1, 3, 17]
        widths = np.array(rng.permutation(widths), dtype=np.int64)
        ops = rng.integers(0, 2, len(widths))
        ops = np.where(ops == 0, C.SOFTMAX, C.RMSNORM)
        flat, rows, _ = packed_batch(widths, ops, dt, seed=dt + 5)
        d_in = flat.cuda()
        d_out = torch.full_like(d_in, float("nan"))
        R = C.Ragged(rows, dt, d_in, d_out, tune=False)
        info = R.info()
        R.run()
        torch.cuda.synchronize()
        assert C.device_error() == C.OK
        check_rows(flat, d_out, rows, dt, range(len(rows)))
        assert not torch.isnan(d_out.float()).any()
        R.close()
        assert info["cluster_size"] == P and info["vector_groups"] == int(force[3])
        assert info["narrow_items"] > 0 and info["huge_items"] > 0
        assert P == 1 or info["wide_items"] > 0


def test_ragged_20000_rows_tuned_sampled_parity():
    widths, ops = synth.ragged_widths(20000, seed=synth.SEED_RAGGED)
    widths, ops = widths.numpy(), ops.numpy()
    dt = C.BF16
    offs = np.concatenate([[0], np.cumsum(widths)[:-1]]).astype(np.int64)
    total = int(widths.sum())
    g = torch.Generator(device="cuda").manual_seed(synth.SEED_DATA)
    d_in = (torch.randn(total, generator=g, device="cuda") * 2.0).to(torch.bfloat16)
    d_out = torch.empty_like(d_in)
    rows = [(int(o), int(o), int(w), int(op)) for o, w, op in zip(offs, widths, ops)]
    R = C.Ragged(rows, dt, d_in, d_out, tune=True)
    info = R.info()
    d_out.fill_(float("nan"))
    R.run()
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    rng = np.random.default_rng(0)
    pick = list(rng.choice(len(rows), 48, replace=False)) + [int(np.argmax(widths)), int(np.argmin(widths))]
    check_rows(d_in.cpu(), d_out, rows, dt, pick)
    assert not torch.isnan(d_out.float()).any()  # every element written
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(5):
        R.run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / 5
    gbs = total * 4 / ms / 1e6
    print(f"ragged 20000 rows BF16: {ms:.3f} ms, {gbs:.0f} GB/s algorithmic, info {info}")
    R.close()
