"""Seeded synthetic inputs for the row ops (shared by tests, bench and smoke).

This module draws random numbers and stores them in the I/O formats; it holds
none of the method's arithmetic (no reduction, no normalisation, no softmax).
The paper's workloads are synthetic FP32 row tensors (Sec. IV-A); the recipes
here follow the workload descriptions the library is measured on:

* ``normal``      x ~ N(0, std^2)
* ``outliers``    x ~ N(0, 1), each element replaced with probability 1% by
                  +50 or -50 (fair sign)
* ``gamma_beta``  gamma ~ N(1, 0.1^2), beta ~ N(0, 0.1^2)
* ``to_e4m3_rowscaled``  per-row scale s = amax|x| / 448 (FP32), codes
                  q = RNE(x / s) saturated to +-448, stored as float8_e4m3fn
* ``ragged_widths``  widths round(2^(10 + 10u)), u ~ U[0, 1); op per row is a
                  fair coin between softmax and RMSNorm
* ``sweep_shapes``   rows round(2^U(6,16)), cols round(2^U(10,20)), dtype and
                  op uniform, resampled while the I/O bytes exceed a cap

Seeds: 0 data, 1 gamma/beta, 2 ragged widths and ops, 3 sweep shapes.
"""
from __future__ import annotations

import math

import torch

SEED_DATA, SEED_AFFINE, SEED_RAGGED, SEED_SWEEP = 0, 1, 2, 3
E4M3_MAX = 448.0


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def normal(rows: int, cols: int, *, std: float = 1.0, seed: int = SEED_DATA,
           device="cpu", mean: float = 0.0) -> torch.Tensor:
    g = _gen(seed, device)
    x = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
    if std != 1.0:
        x.mul_(std)
    if mean != 0.0:
        x.add_(mean)
    return x


def outliers(rows: int, cols: int, *, seed: int = SEED_DATA, device="cpu",
             p: float = 0.01, mag: float = 50.0) -> torch.Tensor:
    g = _gen(seed, device)
    x = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
    u = torch.rand(rows, cols, generator=g, device=device)
    sgn = torch.rand(rows, cols, generator=g, device=device) < 0.5
    val = torch.where(sgn, torch.full_like(x, mag), torch.full_like(x, -mag))
    return torch.where(u < p, val, x)


def gamma_beta(cols: int, *, seed: int = SEED_AFFINE, device="cpu"):
    g = _gen(seed, device)
    gamma = 1.0 + 0.1 * torch.randn(cols, generator=g, device=device, dtype=torch.float32)
    beta = 0.1 * torch.randn(cols, generator=g, device=device, dtype=torch.float32)
    return gamma, beta


def to_bf16(x: torch.Tensor) -> torch.Tensor:
    return x.to(torch.bfloat16)


def to_e4m3_rowscaled(x: torch.Tensor):
    """Per-row scaled FP8-E4M3 codes and the FP32 scales (rows,)."""
    amax = x.abs().amax(dim=1).to(torch.float32)
    scale = torch.where(amax > 0, amax / E4M3_MAX, torch.ones_like(amax))
    q = (x / scale[:, None]).clamp_(-E4M3_MAX, E4M3_MAX).to(torch.float8_e4m3fn)
    return q, scale


def ragged_widths(n_rows: int, *, seed: int = SEED_RAGGED, lo_log2: float = 10.0,
                  hi_log2: float = 20.0):
    """(widths int64 tensor, ops tensor: 0 softmax / 3 rmsnorm)."""
    g = _gen(seed, "cpu")
    u = torch.rand(n_rows, generator=g, dtype=torch.float64)
    w = torch.round(torch.pow(2.0, lo_log2 + (hi_log2 - lo_log2) * u)).to(torch.int64)
    coin = torch.rand(n_rows, generator=g, dtype=torch.float64) < 0.5
    ops = torch.where(coin, torch.zeros(n_rows, dtype=torch.int64),
                      torch.full((n_rows,), 3, dtype=torch.int64))
    return w, ops


def sweep_shapes(n: int, *, seed: int = SEED_SWEEP, cap_bytes: float = 16 * 2**30,
                 rows_log2=(6.0, 16.0), cols_log2=(10.0, 20.0), col_modes=("any",)):
    """List of (op, dtype, rows, cols) with rows*cols*(in+out bytes) <= cap.  Shape i takes its cols as
    drawn when col_modes[i % len(col_modes)] is "any", rounded down to a multiple of 16 for "align16"
    (contiguous rows then start on the 16-byte grid for every dtype), and rounded to the nearest power of
    two for "pow2" (down if that breaks the byte cap)."""
    g = _gen(seed, "cpu")
    size = {0: 4, 1: 2, 2: 1}
    out = []
    while len(out) < n:
        u = torch.rand(4, generator=g, dtype=torch.float64).tolist()
        rows = int(round(2.0 ** (rows_log2[0] + (rows_log2[1] - rows_log2[0]) * u[0])))
        cols = int(round(2.0 ** (cols_log2[0] + (cols_log2[1] - cols_log2[0]) * u[1])))
        dtype = min(2, int(u[2] * 3))
        op = min(3, int(u[3] * 4))
        ob = 4 if op == 1 else size[dtype]
        nbytes = rows * cols * size[dtype] + (rows * 4 if op == 1 else rows * cols * ob)
        if nbytes > cap_bytes:
            continue
        mode = col_modes[len(out) % len(col_modes)]
        if mode == "align16":
            cols = max(16, cols // 16 * 16)
        elif mode == "pow2":
            c2 = 1 << int(round(math.log2(cols)))
            if c2 > cols and rows * c2 * size[dtype] + (rows * 4 if op == 1 else rows * c2 * ob) > cap_bytes:
                c2 //= 2
            cols = c2
        out.append((op, dtype, rows, cols))
    return out


def split_by_shape(n: int, *, seed: int = SEED_SWEEP, train_frac: float = 0.8):
    """Seeded permutation split of n shape indices into (train, held_out)."""
    g = _gen(seed + 1000, "cpu")
    perm = torch.randperm(n, generator=g).tolist()
    k = int(math.floor(train_frac * n))
    return sorted(perm[:k]), sorted(perm[k:])
