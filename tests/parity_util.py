"""Helpers shared by the parity tests: inputs, oracle references, error bounds.

Error bounds (readings of the paper's tolerances):
  FP32 output   softmax: max_i |y - y*| / |y*| <= 1e-5
                logsumexp, layernorm, rmsnorm: max_i |y - y*| / max(|y*|, 1) <= 1e-5
  BF16 output   |y - y*| <= ulp(y*) + e_terms: one BF16 ulp of y*, ulp =
                2^(floor(log2|y*|) - 7) (2^-133 below the normal range).
                softmax, rmsnorm: e_terms = 0 (a product of positive
                factors: the FP32 result is within a few 2^-24 |y*|, and its
                rounding to BF16 adds at most half an ulp).
                layernorm: y* = (x - mu) r g + b can cancel to |y*| << 1, where
                one BF16 ulp is below the rounding error of any FP32
                evaluation of the formula; e_terms = 16 * 2^-24 * ((|x - mu|
                + |mu| + sigma) r |g| + |b|): a few FP32 roundings of each
                term, the |mu| + sigma part for the FP32 error of the mean.
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


LN_TERM_ULPS = 16.0


def ln_terms(x64: np.ndarray, gamma=None, beta=None, eps=None) -> np.ndarray:
    """Per-element magnitude (|x - mu| + |mu| + sigma) r |g| + |b| of the LayerNorm formula's terms, from the
    FP64 row statistics of the decoded input x64 (rows x cols)."""
    eps = 1e-5 if eps is None or eps < 0 else eps
    mu = x64.mean(axis=1, keepdims=True)
    var = ((x64 - mu) ** 2).mean(axis=1, keepdims=True)
    r = 1.0 / np.sqrt(var + eps)
    g = np.ones(x64.shape[1]) if gamma is None else np.abs(np.asarray(gamma, dtype=np.float64))
    b = np.zeros(x64.shape[1]) if beta is None else np.abs(np.asarray(beta, dtype=np.float64))
    return (np.abs(x64 - mu) + np.abs(mu) + np.sqrt(var)) * r * g[None, :] + b[None, :]


def decoded(x_cpu: torch.Tensor, scale=None) -> np.ndarray:
    """The stored input as exact FP64 values (E4M3 codes times their row scale)."""
    x = to64(x_cpu)
    if scale is not None:
        x = x * np.asarray(scale.cpu(), dtype=np.float64).reshape(-1, 1)
    return x


def error_metric(op: int, out_dtype: int, y: np.ndarray, ref: np.ndarray, out_scale=None, *, x64=None, gamma=None,
                 beta=None, eps=None) -> float:
    """Error in units of the bound (<= 1.0 passes).  LayerNorm with BF16 output needs x64 (the decoded input)
    and its gamma / beta / eps for the term bound."""
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
        extra = 0.0
        if op == C.LAYERNORM:
            if x64 is None:
                raise ValueError("LayerNorm BF16 bound needs the decoded input")
            extra = LN_TERM_ULPS * 2.0 ** -24 * ln_terms(x64, gamma, beta, eps)
        return float(np.max(np.abs(y - ref) / (ulp + extra))) if y.size else 0.0
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
    m = error_metric(op, out_dtype, to64(out), ref, None if osc is None else osc.cpu().numpy(),
                     x64=decoded(x_cpu, scale) if op == C.LAYERNORM else None, gamma=gamma, beta=beta,
                     eps=None if eps < 0 else eps)
    assert m <= limit, f"error {m:.3f} x bound (op={op}, in={in_dtype}, out={out_dtype}, plan={plan})"
    return m, out


# ---------------------------------------------------------------- backward ops
BWD_FWD_OP = {C.SOFTMAX_BWD: O.SOFTMAX, C.LAYERNORM_BWD: O.LAYERNORM, C.RMSNORM_BWD: O.RMSNORM,
              C.SOFTMAX_LOGITS_BWD: O.SOFTMAX_LOGITS, C.XENT_BWD: O.XENT}


def bwd_inputs(op: int, dtype: int, rows: int, cols: int, *, ld: int = 0, seed: int = 0, device="cpu"):
    """Tensors (a, dy, gamma, mean, rstd) on `device` for a backward op: a is softmax(N(0, 3^2) logits)
    (softmax), N(0, 3^2) logits (the logits ops) or the outlier-laden x of the forward workload (norms);
    dy ~ N(0, 1), for the cross entropy the targets softmax(N(0, 1)); gamma ~ N(1, 0.1); mean / rstd are
    the FP64 row statistics of the stored a, rounded to FP32 (the forward's saved statistics).  For the
    cross entropy the last entry is the per-row scale w ~ U(0.5, 2) instead of rstd."""
    ld = ld or cols
    if op in (C.SOFTMAX_LOGITS_BWD, C.XENT_BWD):
        a = torch.zeros(rows, ld, dtype=torch.float32, device=device)
        a[:, :cols] = synth.normal(rows, cols, std=3.0, seed=seed, device=device)
        if op == C.XENT_BWD:
            dy = torch.zeros(rows, ld, dtype=torch.float32, device=device)
            dy[:, :cols] = torch.softmax(synth.normal(rows, cols, seed=seed + 1, device=device).double(), 1).float()
            w = 0.5 + 1.5 * torch.rand(rows, generator=torch.Generator(device=device).manual_seed(seed + 3),
                                       device=device)
        else:
            dy = synth.normal(rows, ld, seed=seed + 1, device=device)
        if dtype == C.BF16:
            a, dy = synth.to_bf16(a), synth.to_bf16(dy)
        return a, dy, None, None, (w if op == C.XENT_BWD else None)
    if op == C.SOFTMAX_BWD:
        logits = synth.normal(rows, cols, std=3.0, seed=seed, device=device).double()
        a = torch.zeros(rows, ld, dtype=torch.float32, device=device)
        a[:, :cols] = torch.softmax(logits, dim=1).float()
        del logits
    else:
        a = synth.outliers(rows, ld, seed=seed, device=device)
    dy = synth.normal(rows, ld, seed=seed + 1, device=device)
    if dtype == C.BF16:
        a, dy = synth.to_bf16(a), synth.to_bf16(dy)
    gamma = synth.gamma_beta(cols, seed=seed + 2, device=device)[0] if op != C.SOFTMAX_BWD else None
    mean = rstd = None
    if op != C.SOFTMAX_BWD:
        a64 = a[:, :cols].double()
        if op == C.LAYERNORM_BWD:
            m = a64.mean(dim=1)
            rstd = (1.0 / torch.sqrt(((a64 - m[:, None]) ** 2).mean(dim=1) + 1e-5)).float()
            mean = m.float()
        else:
            rstd = (1.0 / torch.sqrt((a64 * a64).mean(dim=1) + 1e-6)).float()
        del a64
    return a, dy, gamma, mean, rstd


def bwd_reference(op, dtype, a, dy, gamma, mean, rstd, rows, cols, ld=0):
    f = lambda t: None if t is None else t.cpu().numpy()  # noqa: E731
    dx64, _ = O.run_bwd(BWD_FWD_OP[op], dtype, raw_numpy(a), raw_numpy(dy), rows, cols, ld=ld or cols,
                        gamma=f(gamma), mean=f(mean), rstd=f(rstd))  # for the cross entropy rstd is the scale
    return dx64


def bwd_error(op, dtype, dx, ref, a, dy, gamma, mean, rstd, cols):
    """Error of dx (rows x cols, FP64) in units of the bound (<= 1.0 passes).

    The bound is 1e-5 of the row's largest term of the formula, S_row, plus one BF16 ulp of the exact
    value for BF16 output: softmax S = max|y| (max|dy| + sum|y dy|); layernorm S = rstd (max|g| + sum|g|/N
    + max|xh| sum|g xh|/N); rmsnorm S = rstd (max|g| + max|xh| sum|g xh|/N), g = dy gamma.  FP32 sums of N
    terms err by a small multiple of 2^-24 times the sum of the terms' magnitudes; dx cancels, so its error
    is measured against those magnitudes, not against |dx|."""
    a64, dy64 = to64(a)[:, :cols], to64(dy)[:, :cols]
    if op == C.SOFTMAX_BWD:
        S = np.abs(a64).max(axis=1) * (np.abs(dy64).max(axis=1) + np.abs(a64 * dy64).sum(axis=1))
    elif op == C.SOFTMAX_LOGITS_BWD:  # the softmax bound with y recomputed from the logits
        y = O.softmax(a64)
        S = np.abs(y).max(axis=1) * (np.abs(dy64).max(axis=1) + np.abs(y * dy64).sum(axis=1))
    elif op == C.XENT_BWD:  # w (max y |sum t| + max |t|)
        y = O.softmax(a64)
        w = np.ones(a64.shape[0]) if rstd is None else rstd.cpu().double().numpy()
        S = np.abs(w) * (np.abs(y).max(axis=1) * np.abs(dy64.sum(axis=1)) + np.abs(dy64).max(axis=1))
    else:
        g = dy64 * (1.0 if gamma is None else gamma.cpu().double().numpy()[None, :])
        r = rstd.cpu().double().numpy()
        xh = (a64 - (mean.cpu().double().numpy()[:, None] if op == C.LAYERNORM_BWD else 0.0)) * r[:, None]
        S = np.abs(g).max(axis=1) + np.abs(xh).max(axis=1) * np.abs(g * xh).sum(axis=1) / cols
        if op == C.LAYERNORM_BWD:
            S = S + np.abs(g).sum(axis=1) / cols
        S = r * S
    bound = F32_TOL * S[:, None]
    if dtype == C.BF16:
        mag = np.abs(ref)
        ulp = np.where(mag > 0, np.exp2(np.floor(np.log2(np.where(mag > 0, mag, 1.0))) - 7), 2.0 ** -133)
        bound = bound + ulp
    return float((np.abs(dx - ref) / bound).max())


# ---------------------------------------------------------------- two-input statistics (weighted variance, Pearson)
def pair_inputs(op: int, dtype: int, rows: int, cols: int, *, ld: int = 0, seed: int = 0, device="cpu"):
    """Tensors (x, d, g): weighted variance x ~ N(3, 2^2) with 1% +-50 outliers and weights d ~ U(0.1, 2);
    Pearson x with outliers and d = 0.5 x + N(0, 1); per-row upstream gradients g ~ U(0.5, 2)."""
    ld = ld or cols
    x = synth.outliers(rows, ld, seed=seed, device=device)
    gen = torch.Generator(device=device).manual_seed(seed + 7)
    if op == C.WVAR_BWD:
        x = 2.0 * x + 3.0
        d = 0.1 + 1.9 * torch.rand(rows, ld, generator=gen, device=device)
    else:
        d = 0.5 * x + synth.normal(rows, ld, seed=seed + 1, device=device)
    g = 0.5 + 1.5 * torch.rand(rows, generator=gen, device=device)
    if dtype == C.BF16:
        x, d = synth.to_bf16(x), synth.to_bf16(d)
    return x, d, g


def pair_reference(op, x, d, g, cols):
    x64, d64 = to64(x)[:, :cols], to64(d)[:, :cols]
    gg = g.cpu().double().numpy()
    return O.wvar_bwd(x64, d64, gg) if op == C.WVAR_BWD else O.pearson_bwd(x64, d64, gg)


def pair_error(op, dtype, out1, out2, ref1, ref2, x, d, g, cols):
    """Largest error of the two gradients in units of their bounds (<= 1.0 passes): 1e-5 of the row's
    largest term of each formula, plus one BF16 ulp of the exact value for BF16.  Weighted variance: dx terms
    g 2 w (x - mu) / W, dw terms g (x - mu)^2 / W and g v / W; Pearson: g (y - yb) / sqrt(Sxx Syy) and
    g r (x - xb) / Sxx (dx), symmetrically for dy.  The bound depends only on the exact values of the terms
    (FP64, from the inputs), not on how a kernel accumulates the moments."""
    x64, d64 = to64(x)[:, :cols], to64(d)[:, :cols]
    gg = np.abs(g.cpu().double().numpy())
    if op == C.WVAR_BWD:
        W = d64.sum(axis=1)
        mu = (d64 * x64).sum(axis=1) / W
        u = x64 - mu[:, None]
        v = (d64 * u * u).sum(axis=1) / W
        S1 = gg / W * np.abs(2 * d64 * u).max(axis=1)
        S2 = gg / W * ((u * u).max(axis=1) + v)
    else:
        u = x64 - x64.mean(axis=1, keepdims=True)
        w_ = d64 - d64.mean(axis=1, keepdims=True)
        sxx, syy = (u * u).sum(axis=1), (w_ * w_).sum(axis=1)
        den = np.sqrt(sxx * syy)
        r = np.abs((u * w_).sum(axis=1)) / den
        S1 = gg * (np.abs(w_).max(axis=1) / den + r * np.abs(u).max(axis=1) / sxx)
        S2 = gg * (np.abs(u).max(axis=1) / den + r * np.abs(w_).max(axis=1) / syy)
    worst = 0.0
    for out, ref, S in ((out1, ref1, S1), (out2, ref2, S2)):
        bound = F32_TOL * S[:, None]
        if dtype == C.BF16:
            mag = np.abs(ref)
            bound = bound + np.where(mag > 0, np.exp2(np.floor(np.log2(np.where(mag > 0, mag, 1.0))) - 7), 2.0 ** -133)
        e = np.abs(out - ref) / bound
        if not np.all(np.isfinite(e)):  # a NaN or infinite output fails (max() would skip a NaN)
            return float("inf")
        worst = max(worst, float(e.max()))
    return worst
