"""FP64 CPU oracle for the CREDIT reduction-reuse row ops.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_2609_01864_gb300``) never imports it, and it never imports the product
library: the two share no code and meet only at the seeded input bytes.

Contents
--------
* ``credit_oracle.c`` -- the plain double-precision definitions of softmax,
  log-sum-exp, LayerNorm and RMSNorm (Eq. 1 of the paper, one row at a time)
  and of the input gradients of softmax, LayerNorm and RMSNorm (the backward
  members of the workload suite, Sec. IV-A),
  exact decoding of BF16 / FP8-E4M3 inputs and round-to-nearest-even encoding
  of BF16 / E4M3 outputs, written from the formats' definitions.
* ``cost_model`` -- the analytic profitability model (Eq. 3, 4, 6-9).
* ``mlp`` -- FP64 forward / backward / Adam of the latency MLP.

The C part is compiled with gcc on first use (or by ``build()``) into
``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "credit_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

F32, BF16, E4M3 = 0, 1, 2
SOFTMAX, LOGSUMEXP, LAYERNORM, RMSNORM = 0, 1, 2, 3
SOFTMAX_LOGITS, XENT = 7, 8  # backward ops from logits (run_bwd only)
DTYPE_SIZE = {F32: 4, BF16: 2, E4M3: 1}
E4M3_MAX = 448.0


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, OpenMP, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            so = build()
            L = ctypes.CDLL(so)
            d, i64, vp, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int
            L.oracle_bf16_to_double.restype = d
            L.oracle_bf16_to_double.argtypes = [ctypes.c_uint16]
            L.oracle_e4m3_to_double.restype = d
            L.oracle_e4m3_to_double.argtypes = [ctypes.c_uint8]
            L.oracle_double_to_bf16.restype = ctypes.c_uint16
            L.oracle_double_to_bf16.argtypes = [d]
            L.oracle_double_to_e4m3_sat.restype = ctypes.c_uint8
            L.oracle_double_to_e4m3_sat.argtypes = [d]
            L.oracle_softmax_row.argtypes = [vp, i64, vp]
            L.oracle_lse_row.restype = d
            L.oracle_lse_row.argtypes = [vp, i64]
            L.oracle_layernorm_row.argtypes = [vp, i64, vp, vp, d, vp]
            L.oracle_rmsnorm_row.argtypes = [vp, i64, vp, d, vp]
            L.oracle_decode.argtypes = [i32, vp, vp, i64, i64, i64, vp]
            L.oracle_run.restype = i32
            L.oracle_run.argtypes = [i32, i32, i32, vp, vp, i64, i64, i64, vp, vp, d,
                                     vp, vp, i64, vp, i32]
            L.oracle_softmax_bwd_row.argtypes = [vp, vp, i64, vp]
            L.oracle_layernorm_bwd_row.argtypes = [vp, vp, i64, vp, d, d, vp]
            L.oracle_rmsnorm_bwd_row.argtypes = [vp, vp, i64, vp, d, vp]
            L.oracle_softmax_logits_bwd_row.argtypes = [vp, vp, i64, vp]
            L.oracle_xent_bwd_row.argtypes = [vp, vp, i64, d, vp]
            L.oracle_wvar_row.restype = d
            L.oracle_wvar_row.argtypes = [vp, vp, i64]
            L.oracle_wvar_bwd_row.argtypes = [vp, vp, i64, d, vp, vp]
            L.oracle_pearson_row.restype = d
            L.oracle_pearson_row.argtypes = [vp, vp, i64]
            L.oracle_pearson_bwd_row.argtypes = [vp, vp, i64, d, vp, vp]
            L.oracle_scan_row.argtypes = [vp, i64, vp]
            L.oracle_stencil_row.argtypes = [vp, i64, vp, i32, vp]
            L.oracle_quant_int8_row.restype = ctypes.c_float
            L.oracle_quant_int8_row.argtypes = [vp, i64, vp]
            L.oracle_run_bwd.restype = i32
            L.oracle_run_bwd.argtypes = [i32, i32, vp, vp, i64, i64, i64, vp, vp, vp, vp, vp, i32]
            L.oracle_max_threads.restype = i32
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- formats
def bf16_to_double(codes: np.ndarray) -> np.ndarray:
    L = lib()
    c = np.asarray(codes, dtype=np.uint16).ravel()
    return np.array([L.oracle_bf16_to_double(int(v)) for v in c]).reshape(np.shape(codes))


def e4m3_to_double(codes: np.ndarray) -> np.ndarray:
    L = lib()
    c = np.asarray(codes, dtype=np.uint8).ravel()
    return np.array([L.oracle_e4m3_to_double(int(v)) for v in c]).reshape(np.shape(codes))


def double_to_bf16(v: np.ndarray) -> np.ndarray:
    L = lib()
    a = np.asarray(v, dtype=np.float64).ravel()
    return np.array([L.oracle_double_to_bf16(float(x)) for x in a], dtype=np.uint16).reshape(np.shape(v))


def double_to_e4m3(v: np.ndarray) -> np.ndarray:
    L = lib()
    a = np.asarray(v, dtype=np.float64).ravel()
    return np.array([L.oracle_double_to_e4m3_sat(float(x)) for x in a], dtype=np.uint8).reshape(np.shape(v))


# ---------------------------------------------------------------- row ops
def softmax(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_softmax_row(_ptr(x[r]), x.shape[1], _ptr(y[r]))
    return y


def logsumexp(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    return np.array([lib().oracle_lse_row(_ptr(x[r]), x.shape[1]) for r in range(x.shape[0])])


def layernorm(x, gamma=None, beta=None, eps=1e-5):
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
    y = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_layernorm_row(_ptr(x[r]), x.shape[1], _ptr(g), _ptr(b), eps, _ptr(y[r]))
    return y


def rmsnorm(x, gamma=None, eps=1e-6):
    x = np.ascontiguousarray(x, dtype=np.float64)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    y = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_rmsnorm_row(_ptr(x[r]), x.shape[1], _ptr(g), eps, _ptr(y[r]))
    return y


def decode(dtype: int, raw: np.ndarray, rows: int, cols: int, ld: int = 0, in_scale=None) -> np.ndarray:
    """Exact FP64 values of `rows` x `cols` stored elements (raw: bytes/words)."""
    raw = np.ascontiguousarray(raw)
    sc = None if in_scale is None else np.ascontiguousarray(in_scale, dtype=np.float32)
    x = np.empty((rows, cols), dtype=np.float64)
    lib().oracle_decode(dtype, _ptr(raw), _ptr(sc), rows, cols, ld or cols, _ptr(x))
    return x


DEFAULT_EPS = {SOFTMAX: 0.0, LOGSUMEXP: 0.0, LAYERNORM: 1e-5, RMSNORM: 1e-6}


def run(op: int, in_dtype: int, raw: np.ndarray, rows: int, cols: int, *, out_dtype=None,
        in_scale=None, gamma=None, beta=None, eps=None, ld_in: int = 0,
        want_exact: bool = True, want_encoded: bool = False, nthreads: int = 0):
    """Batch oracle.  Returns (y64 or None, encoded or None, out_scale or None).

    raw holds the stored input elements (float32 / uint16 bf16 codes / uint8
    e4m3 codes).  y64 is (rows, cols) or (rows,) for log-sum-exp.
    """
    out_dtype = in_dtype if out_dtype is None else out_dtype
    if op == LOGSUMEXP:
        out_dtype = F32
    eps = DEFAULT_EPS[op] if eps is None else eps
    raw = np.ascontiguousarray(raw)
    sc = None if in_scale is None else np.ascontiguousarray(in_scale, dtype=np.float32)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float32)
    b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float32)
    shape = (rows,) if op == LOGSUMEXP else (rows, cols)
    y64 = np.empty(shape, dtype=np.float64) if want_exact else None
    enc = None
    osc = None
    if want_encoded:
        npdt = {F32: np.float32, BF16: np.uint16, E4M3: np.uint8}[out_dtype]
        enc = np.empty(shape, dtype=npdt)
        if out_dtype == E4M3:
            osc = np.empty(rows, dtype=np.float32)
    rc = lib().oracle_run(op, in_dtype, out_dtype, _ptr(raw), _ptr(sc), rows, cols, ld_in,
                          _ptr(g), _ptr(b), float(eps), _ptr(y64), _ptr(enc),
                          0 if op == LOGSUMEXP else cols, _ptr(osc), nthreads)
    if rc != 0:
        raise ValueError("oracle_run rejected its arguments")
    return y64, enc, osc


# ---------------------------------------------------------------- input gradients
def softmax_bwd(y, dy):
    """dx of softmax given its output y and the upstream gradient dy (rows x cols, FP64)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    dx = np.empty_like(y)
    for r in range(y.shape[0]):
        lib().oracle_softmax_bwd_row(_ptr(y[r]), _ptr(dy[r]), y.shape[1], _ptr(dx[r]))
    return dx


def layernorm_bwd(x, dy, mean, rstd, gamma=None):
    """dx of LayerNorm given its input x, dy and the saved per-row mean / rstd (FP64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    dx = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_layernorm_bwd_row(_ptr(x[r]), _ptr(dy[r]), x.shape[1], _ptr(g), float(mean[r]),
                                       float(rstd[r]), _ptr(dx[r]))
    return dx


def rmsnorm_bwd(x, dy, rstd, gamma=None):
    """dx of RMSNorm given its input x, dy and the saved per-row rstd (FP64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    g = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
    dx = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_rmsnorm_bwd_row(_ptr(x[r]), _ptr(dy[r]), x.shape[1], _ptr(g), float(rstd[r]), _ptr(dx[r]))
    return dx


def softmax_logits_bwd(z, dy):
    """dz of softmax given its logits z (the output is recomputed) and the upstream gradient dy (FP64)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    dy = np.ascontiguousarray(dy, dtype=np.float64)
    dz = np.empty_like(z)
    for r in range(z.shape[0]):
        lib().oracle_softmax_logits_bwd_row(_ptr(z[r]), _ptr(dy[r]), z.shape[1], _ptr(dz[r]))
    return dz


def xent_bwd(z, t, w=None):
    """dz of the cross entropy -sum t log softmax(z) per row, times the row scale w (None = 1) (FP64)."""
    z = np.ascontiguousarray(z, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    dz = np.empty_like(z)
    for r in range(z.shape[0]):
        lib().oracle_xent_bwd_row(_ptr(z[r]), _ptr(t[r]), z.shape[1], 1.0 if w is None else float(w[r]), _ptr(dz[r]))
    return dz


def _pair_rows(a, b):
    return np.ascontiguousarray(a, dtype=np.float64), np.ascontiguousarray(b, dtype=np.float64)


def wvar(x, w):
    """Weighted variance sum w (x - mu)^2 / sum w per row, mu = sum w x / sum w (FP64)."""
    x, w = _pair_rows(x, w)
    return np.array([lib().oracle_wvar_row(_ptr(x[r]), _ptr(w[r]), x.shape[1]) for r in range(x.shape[0])])


def wvar_bwd(x, w, g=None):
    """(dx, dw) of the weighted variance times the per-row upstream gradient g (None = 1) (FP64)."""
    x, w = _pair_rows(x, w)
    dx, dw = np.empty_like(x), np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_wvar_bwd_row(_ptr(x[r]), _ptr(w[r]), x.shape[1], 1.0 if g is None else float(g[r]),
                                  _ptr(dx[r]), _ptr(dw[r]))
    return dx, dw


def pearson(x, y):
    """Pearson correlation of x and y per row (FP64)."""
    x, y = _pair_rows(x, y)
    return np.array([lib().oracle_pearson_row(_ptr(x[r]), _ptr(y[r]), x.shape[1]) for r in range(x.shape[0])])


def pearson_bwd(x, y, g=None):
    """(dx, dy) of the Pearson correlation times the per-row upstream gradient g (None = 1) (FP64)."""
    x, y = _pair_rows(x, y)
    dx, dy = np.empty_like(x), np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_pearson_bwd_row(_ptr(x[r]), _ptr(y[r]), x.shape[1], 1.0 if g is None else float(g[r]),
                                     _ptr(dx[r]), _ptr(dy[r]))
    return dx, dy


def run_bwd(op: int, dtype: int, a_raw, dy_raw, rows: int, cols: int, *, gamma=None, mean=None, rstd=None,
            ld: int = 0, want_exact: bool = True, want_encoded: bool = False, nthreads: int = 0):
    """Batch input gradient.  op is the forward op (SOFTMAX, LAYERNORM, RMSNORM) or SOFTMAX_LOGITS / XENT;
    a_raw is the forward output (softmax), input (norms) or the logits (SOFTMAX_LOGITS, XENT), dy_raw the
    upstream gradient (XENT: the target weights), both stored elements of dtype (F32 / BF16 codes) with row
    stride ld; gamma, mean, rstd (XENT: the per-row upstream scale) are FP32 arrays.  Returns (dx64 or None,
    encoded or None)."""
    a_raw = np.ascontiguousarray(a_raw)
    dy_raw = np.ascontiguousarray(dy_raw)
    f32 = lambda v: None if v is None else np.ascontiguousarray(v, dtype=np.float32)  # noqa: E731
    g, mu, rs = f32(gamma), f32(mean), f32(rstd)
    dx64 = np.empty((rows, cols), dtype=np.float64) if want_exact else None
    enc = None
    if want_encoded:
        enc = np.empty((rows, ld or cols), dtype={F32: np.float32, BF16: np.uint16}[dtype])
    rc = lib().oracle_run_bwd(op, dtype, _ptr(a_raw), _ptr(dy_raw), rows, cols, ld, _ptr(g), _ptr(mu), _ptr(rs),
                              _ptr(dx64), _ptr(enc), nthreads)
    if rc != 0:
        raise ValueError("oracle_run_bwd rejected its arguments")
    return dx64, (None if enc is None else enc[:, :cols])


def quant_int8(x):
    """Row-wise int8 quantisation of FP32 rows: (codes int8, scales float32)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.empty(x.shape, dtype=np.int8)
    s = np.empty(x.shape[0], dtype=np.float32)
    for r in range(x.shape[0]):
        s[r] = lib().oracle_quant_int8_row(_ptr(x[r]), x.shape[1], _ptr(q[r]))
    return q, s


def scan(x):
    """Row-wise inclusive prefix sums (FP64) of rows x (rows x cols)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    for r in range(x.shape[0]):
        lib().oracle_scan_row(_ptr(x[r]), x.shape[1], _ptr(y[r]))
    return y


def stencil(x, w):
    """Row-wise stencil with weights w (2r + 1 of them, radius r), zero padding at the row ends (FP64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    y = np.empty_like(x)
    r = (len(w) - 1) // 2
    for i in range(x.shape[0]):
        lib().oracle_stencil_row(_ptr(x[i]), x.shape[1], _ptr(w), r, _ptr(y[i]))
    return y


def max_threads() -> int:
    return int(lib().oracle_max_threads())
