"""Helpers shared by the parity tests: inputs, oracle references, error bounds.

Error bounds (the readings are listed in the design doc):
  FP32 output   softmax: max_i |y - y*| / |y*| <= 1e-5
                logsumexp, layernorm, rmsnorm: max_i |y - y*| / max(|y*|, 1) <= 1e-5
  BF16 output   |y - y*| <= ulp(y*) + e32(y*): one BF16 ulp of y*, ulp =
                2^(floor(log2|y*|) - 7) (2^-133 below the normal range), on
                top of the FP32 bound e32 (1e-5 |y*| for softmax, 1e-5
                max(|y*|, 1) otherwise).  Without e32 the bound cannot be met
                with FP32 statistics where the normalised output cancels to
                |y*| << 1 (LayerNorm with beta).
  FP8 output    |q * s - y*| <= 2^(max(floor(log2(|y*| / s)), -6) - 3) * s, one
                E4M3 quantum at the scaled value, and s within 1e-5 (relative)
                of amax|y*| / 448
"""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from paper_2609_01864_gb300 import credit as C
from paper_2609_01864_gb300 import synth

F32_TOL = 1e-5


def make_input(dtype: int, rows: int, cols: int, *, kind: str = "normal", std: float = 1.0, seed: int = 0,
               mean: float = 0.0):
    """CPU tensors: (stored input, per-row FP32 scale or None)."""
    if kind == "outliers":
        x = synth.outliers(rows, cols, seed=seed)
    else:
        x = synth.normal(rows, cols, std=std, seed=seed, mean=mean)
    if dtype == C.F32:
        return x, None
    if dtype == C.BF16:
        return synth.to_bf16(x), None
    q, s = synth.to_e4m3_rowscaled(x)
    return q, s


def raw_numpy(t: torch.Tensor) -> np.ndarray:
    t = t.detach().cpu().contiguous()
    if t.dtype == torch.float32:
        return t.numpy()
    if t.dtype == torch.bfloat16:
        return t.view(torch.int16).numpy().view(np.uint16)
    if t.dtype == torch.float8_e4m3fn:
        return t.view(torch.uint8).numpy()
    raise TypeError(t.dtype)


def reference(op: int, in_dtype: int, x_cpu: torch.Tensor, scale=None, gamma=None, beta=None, eps=None):
    rows, cols = x_cpu.shape
    y64, _, _ = O.run(op, in_dtype, raw_numpy(x_cpu), rows, cols,
                      in_scale=None if scale is None else scale.numpy(),
                      gamma=None if gamma is None else gamma.cpu().numpy(),
                      beta=None if beta is None else beta.cpu().numpy(), eps=eps)
    return y64


def to64(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().to(torch.float64).numpy()


def error_metric(op: int, out_dtype: int, y: np.ndarray, ref: np.ndarray, out_scale=None) -> float:
    """Error in units of the bound (<= 1.0 passes)."""
    if op == C.LOGSUMEXP or out_dtype == C.F32:
        if op == C.SOFTMAX:
            den = np.abs(ref)
            den = np.where(den > 0, den, 1.0)
        else:
            den = np.maximum(np.abs(ref), 1.0)
        return float(np.max(np.abs(y - ref) / den) / F32_TOL) if y.size else 0.0
    if out_dtype == C.BF16:
        a = np.abs(ref)
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
        ulp = np.where(a >= 2.0 ** -126, np.exp2(e - 7), 2.0 ** -133)
        e32 = F32_TOL * (a if op == C.SOFTMAX else np.maximum(a, 1.0))
        return float(np.max(np.abs(y - ref) / (ulp + e32))) if y.size else 0.0
    # FP8: y holds decoded codes (not yet scaled)
    s = np.asarray(out_scale, dtype=np.float64).reshape(-1, 1)
    t = np.abs(ref) / s
    e = np.floor(np.log2(np.where(t > 0, t, 2.0 ** -30)))
    q = np.exp2(np.maximum(e, -6) - 3) * s
    err = float(np.max(np.abs(y * s - ref) / q)) if y.size else 0.0
    amax = np.max(np.abs(ref), axis=1, keepdims=True)
    s_ref = np.where(amax > 0, amax / 448.0, 1.0)
    s_err = float(np.max(np.abs(s - s_ref) / s_ref)) / 1e-5
    return max(err, s_err)


def run_gpu(op, x_cpu, scale, *, out_dtype=None, plan=None, gamma=None, beta=None, eps=-1.0, device="cuda"):
    """Run one op through the C ABI; returns (out tensor on device, out_scale or None)."""
    in_dtype = C.DTYPE_OF[x_cpu.dtype]
    if out_dtype is None:
        out_dtype = C.F32 if op == C.LOGSUMEXP else in_dtype
    x = x_cpu.to(device)
    rows, cols = x.shape
    if op == C.LOGSUMEXP:
        out = torch.empty(rows, device=device, dtype=torch.float32)
    else:
        out = torch.empty(rows, cols, device=device, dtype=C.TORCH_DTYPE[out_dtype])
    osc = torch.empty(rows, device=device, dtype=torch.float32) if (out_dtype == C.FP8_E4M3 and op != C.LOGSUMEXP) else None
    sc = None if scale is None else scale.to(device)
    g = None if gamma is None else gamma.to(device)
    b = None if beta is None else beta.to(device)
    kw = dict(in_dtype=in_dtype, out_dtype=out_dtype, in_scale=sc, out_scale=osc, gamma=g, beta=b, eps=eps)
    if plan is not None and C.plan_check(op, x, out, plan, **kw) == C.ERR_UNSUPPORTED:
        # Only a staged slice too large for one CTA's shared memory (Eq. 3)
        # may be refused; the call must then refuse too, launching nothing.
        assert plan.path in (C.PATH_ONE_CTA, C.PATH_CLUSTER), "two-pass plan refused"
        P = 1 if plan.path == C.PATH_ONE_CTA else plan.cluster_size
        isz = x.element_size()
        body = -(-((cols * isz) // 16) // P) * 16
        assert body > C.slice_capacity(C.FP8_E4M3) - 16 * 16, "legal slice refused"
        n0 = C.launch_count()
        assert C.run_ex_status(op, x, out, plan=plan, **kw) == C.ERR_UNSUPPORTED
        assert C.launch_count() == n0
        return None, None
    C.run_ex(op, x, out, plan=plan, **kw)
    return out, osc


def check_against_oracle(op, x_cpu, scale, *, out_dtype=None, plan=None, gamma=None, beta=None, eps=-1.0,
                         limit: float = 1.0):
    in_dtype = C.DTYPE_OF[x_cpu.dtype]
    if out_dtype is None:
        out_dtype = C.F32 if op == C.LOGSUMEXP else in_dtype
    out, osc = run_gpu(op, x_cpu, scale, out_dtype=out_dtype, plan=plan, gamma=gamma, beta=beta, eps=eps)
    if out is None:
        return None, None
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    ref = reference(op, in_dtype, x_cpu, scale, gamma, beta, None if eps < 0 else eps)
    m = error_metric(op, out_dtype, to64(out), ref, None if osc is None else osc.cpu().numpy())
    assert m <= limit, f"error {m:.3f} x bound (op={op}, in={in_dtype}, out={out_dtype}, plan={plan})"
    return m, out
