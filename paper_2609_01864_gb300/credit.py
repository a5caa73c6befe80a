"""Thin ctypes binding of libcredit.so (include/credit.h).

Argument marshalling only: every step of every op runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (PyTorch supplies device memory and
streams); raw device addresses are accepted where a tensor is.  If the
library is not built the first call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libcredit.so")

# enums of credit.h
F32, BF16, FP8_E4M3, INT8 = 0, 1, 2, 3
SOFTMAX, LOGSUMEXP, LAYERNORM, RMSNORM = 0, 1, 2, 3
QUANT_INT8 = 11
SCAN, STENCIL, SELECT = 12, 13, 14
SCREEN_CANDIDATE, SCREEN_NO_REUSE, SCREEN_ORDERED, SCREEN_REMOTE_STATE = 0, 1, 2, 3
PATH_AUTO, PATH_ONE_CTA, PATH_TWO_PASS, PATH_CLUSTER = -1, 0, 1, 2
OK, ERR_INVALID_ARG, ERR_UNSUPPORTED, ERR_CUDA, ERR_TIMEOUT, ERR_NOT_INITIALIZED, ERR_CAPTURE, ERR_IO = range(8)
OP_NAMES = {SOFTMAX: "softmax", LOGSUMEXP: "logsumexp", LAYERNORM: "layernorm", RMSNORM: "rmsnorm"}
PATH_NAMES = {PATH_ONE_CTA: "one_cta", PATH_TWO_PASS: "two_pass", PATH_CLUSTER: "cluster"}
RETAIN_AUTO, RETAIN_SMEM, RETAIN_TMEM = 0, 1, 2
SOFTMAX_BWD, LAYERNORM_BWD, RMSNORM_BWD, SOFTMAX_LOGITS_BWD, XENT_BWD, WVAR_BWD, PEARSON_BWD = 4, 5, 6, 7, 8, 9, 10
OP_NAMES.update({SOFTMAX_BWD: "softmax_bwd", LAYERNORM_BWD: "layernorm_bwd", RMSNORM_BWD: "rmsnorm_bwd",
                 SOFTMAX_LOGITS_BWD: "softmax_logits_bwd", XENT_BWD: "xent_bwd", WVAR_BWD: "wvar_bwd",
                 PEARSON_BWD: "pearson_bwd"})

TORCH_DTYPE = {F32: torch.float32, BF16: torch.bfloat16, FP8_E4M3: torch.float8_e4m3fn, INT8: torch.int8}
DTYPE_OF = {torch.float32: F32, torch.bfloat16: BF16, torch.float8_e4m3fn: FP8_E4M3, torch.int8: INT8}


class CreditError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


class PlanT(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("cluster_size", ctypes.c_int32), ("ctas_per_row", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ring_chunks", ctypes.c_int32), ("chunk_bytes", ctypes.c_int32),
                ("reducer_threads", ctypes.c_int32), ("retain", ctypes.c_int32), ("smem_bytes", ctypes.c_int64), ("predicted_us", ctypes.c_float), ("source", ctypes.c_int32),
                ("fill_share", ctypes.c_float), ("fill_g", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

    def __repr__(self):
        return f"PlanT({self.as_dict()})"


class ArgsT(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld_in", ctypes.c_int64),
                ("ld_out", ctypes.c_int64), ("in_dtype", ctypes.c_int32), ("out_dtype", ctypes.c_int32),
                ("in_scale", ctypes.c_void_p), ("out_scale", ctypes.c_void_p), ("gamma", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("eps", ctypes.c_float)]


class BwdArgsT(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("dtype", ctypes.c_int32), ("a", ctypes.c_void_p), ("dy", ctypes.c_void_p),
                ("dx", ctypes.c_void_p), ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("gamma", ctypes.c_void_p), ("mean", ctypes.c_void_p), ("rstd", ctypes.c_void_p),
                ("scale", ctypes.c_void_p), ("dx2", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib() -> ctypes.CDLL:
    """Load libcredit.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libcredit.so is not built ({LIB_PATH}); run "
                                   "paper_2609_01864_gb300.build.build() -- there is no fallback path")
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
            L.credit_status_string.restype = ctypes.c_char_p
            L.credit_status_string.argtypes = [i32]
            L.credit_version.restype = i32
            L.credit_init.restype = i32
            L.credit_init.argtypes = [i32]
            for name in ("credit_softmax", "credit_logsumexp", "credit_layernorm", "credit_rmsnorm"):
                f = getattr(L, name)
                f.restype = i32
                f.argtypes = [vp, vp, i64, i64, i32, vp]
            L.credit_plan.restype = i32
            L.credit_plan.argtypes = [i32, i64, i64, i32, ctypes.POINTER(PlanT)]
            L.credit_plan_ex.restype = i32
            L.credit_plan_ex.argtypes = [i32, i64, i64, i32, i32, ctypes.POINTER(PlanT)]
            L.credit_run_ex.restype = i32
            L.credit_run_ex.argtypes = [ctypes.POINTER(ArgsT), ctypes.POINTER(PlanT), vp]
            L.credit_run_host.restype = i32
            L.credit_run_host.argtypes = [ctypes.POINTER(ArgsT), ctypes.POINTER(PlanT)]
            L.credit_run_two_pass_noalloc.restype = i32
            L.credit_run_two_pass_noalloc.argtypes = [ctypes.POINTER(ArgsT), i32, vp]
            L.credit_set_trace.restype = i32
            L.credit_set_trace.argtypes = [vp, i64]
            L.credit_plan_check.restype = i32
            L.credit_plan_check.argtypes = [ctypes.POINTER(ArgsT), ctypes.POINTER(PlanT)]
            L.credit_max_clusters.restype = i32
            L.credit_max_clusters.argtypes = [ctypes.POINTER(ArgsT), ctypes.POINTER(PlanT)]
            L.credit_device_error.restype = i32
            L.credit_device_error.argtypes = [vp]
            L.credit_slice_capacity.restype = i64
            L.credit_slice_capacity.argtypes = [i32]
            L.credit_run_bwd.restype = i32
            L.credit_run_bwd.argtypes = [ctypes.POINTER(BwdArgsT), ctypes.POINTER(PlanT), vp]
            L.credit_plan_bwd.restype = i32
            L.credit_plan_bwd.argtypes = [i32, i64, i64, i32, ctypes.POINTER(PlanT)]
            L.credit_bwd_plan_check.restype = i32
            L.credit_bwd_plan_check.argtypes = [ctypes.POINTER(BwdArgsT), ctypes.POINTER(PlanT)]
            L.credit_launch_count.restype = ctypes.c_longlong
            L.credit_launch_count.argtypes = []
            _extra_prototypes(L)
            _lib = L
    return _lib


class MicrobenchT(ctypes.Structure):
    _fields_ = [("lat_local_cycles", ctypes.c_double), ("lat_remote_cycles", ctypes.c_double),
                ("sync_cycles", ctypes.c_double * 4), ("rate_local_read", ctypes.c_double),
                ("rate_local_store", ctypes.c_double), ("rate_remote_read", ctypes.c_double),
                ("rate_remote_store", ctypes.c_double * 4), ("sm_clock_mhz", ctypes.c_double),
                ("distinct_sms", ctypes.c_int32)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if hasattr(v, "__len__") else v
        return d


class RaggedRowT(ctypes.Structure):
    _fields_ = [("in_off", ctypes.c_int64), ("out_off", ctypes.c_int64), ("cols", ctypes.c_int64),
                ("op", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class RaggedInfoT(ctypes.Structure):
    _fields_ = [("cluster_size", ctypes.c_int32), ("threads", ctypes.c_int32), ("staging_bytes", ctypes.c_int32),
                ("clusters", ctypes.c_int32), ("items", ctypes.c_int64), ("narrow_items", ctypes.c_int64),
                ("wide_items", ctypes.c_int64), ("huge_items", ctypes.c_int64), ("tuned_us", ctypes.c_float),
                ("vector_groups", ctypes.c_int32)]


MODEL_IN_FIELDS = ["M", "N", "P", "T_B_us", "T_ctrl_us", "b_B", "b_reread", "b_keep", "b_in", "s_bytes", "q_sum",
                   "active_clusters", "f_mhz", "B_smem_read", "B_smem_store", "B_dsm_store", "B_peak_gbs"]
MODEL_OUT_FIELDS = ["W", "B_eff_gbs", "T_save_us", "T_replay_us", "T_dsm_us", "T_deposit_us", "T_smem_w_us",
                    "T_input_us", "dT_us"]


class ModelInT(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in MODEL_IN_FIELDS] + [("ablation", ctypes.c_int32)]


class DataflowT(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int32), ("ordered", ctypes.c_int32), ("q_sum", ctypes.c_double),
                ("b_reread", ctypes.c_double), ("remote_bytes_per_elem", ctypes.c_double)]


class ModelOutT(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in MODEL_OUT_FIELDS]


def _extra_prototypes(L):
    """Prototypes of the optional subsystems (profiling, model, ragged, MLP)."""
    i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    L.credit_microbench.restype = i32
    L.credit_microbench.argtypes = [ctypes.POINTER(MicrobenchT), i32]
    L.credit_control_time.restype = i32
    L.credit_control_time.argtypes = [i32, i64, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_float)]
    L.credit_model_eval.restype = i32
    L.credit_model_eval.argtypes = [ctypes.POINTER(ModelInT), ctypes.POINTER(ModelOutT)]
    L.credit_calibrate.restype = i32
    L.credit_calibrate.argtypes = [ctypes.c_char_p, i64]
    L.credit_load_model.restype = i32
    L.credit_load_model.argtypes = [ctypes.c_char_p]
    fp = ctypes.POINTER(ctypes.c_float)
    L.credit_mlp_num_params.restype = i64
    L.credit_mlp_features.restype = i32
    L.credit_mlp_features.argtypes = [i32, i32, i32, i64, i64, i32, i32, i32, i32, ctypes.c_float, fp]
    L.credit_mlp_train.restype = i32
    L.credit_mlp_train.argtypes = [fp, fp, i64, i32, i32, ctypes.c_float, ctypes.c_uint64, fp]
    L.credit_mlp_train_ensemble.restype = i32
    L.credit_mlp_train_ensemble.argtypes = [fp, fp, i64, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, fp]
    L.credit_mlp_members.restype = i32
    L.credit_mlp_members.argtypes = []
    L.credit_mlp_predict.restype = i32
    L.credit_mlp_predict.argtypes = [fp, i64, fp]
    L.credit_mlp_grad.restype = i32
    L.credit_mlp_grad.argtypes = [fp, fp, fp, i64, fp, fp]
    L.credit_dataflow_of.restype = i32
    L.credit_dataflow_of.argtypes = [i32, i32, ctypes.POINTER(DataflowT)]
    L.credit_screen.restype = i32
    L.credit_screen.argtypes = [ctypes.POINTER(DataflowT), i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.credit_plan_control.restype = i32
    L.credit_plan_control.argtypes = [i32, i64, i64, ctypes.POINTER(PlanT), ctypes.POINTER(i32)]
    L.credit_run_control.restype = i32
    L.credit_run_control.argtypes = [i32, vp, vp, i64, i64, i64, i64, vp, i32, vp]
    L.credit_set_wait_test.restype = i32
    L.credit_set_wait_test.argtypes = [i64, i32]
    L.credit_mlp_adam_step.restype = i32
    L.credit_mlp_adam_step.argtypes = [fp, fp, fp, fp, i32, ctypes.c_float]
    L.credit_mlp_save.restype = i32
    L.credit_mlp_save.argtypes = [ctypes.c_char_p]
    L.credit_mlp_load.restype = i32
    L.credit_mlp_load.argtypes = [ctypes.c_char_p]
    L.credit_ragged_create.restype = i32
    L.credit_ragged_create.argtypes = [ctypes.POINTER(RaggedRowT), i64, i32, vp, vp, i32, ctypes.POINTER(vp)]
    L.credit_ragged_run.restype = i32
    L.credit_ragged_run.argtypes = [vp, vp]
    L.credit_ragged_info.restype = i32
    L.credit_ragged_info.argtypes = [vp, ctypes.POINTER(RaggedInfoT)]
    L.credit_ragged_destroy.restype = None
    L.credit_ragged_destroy.argtypes = [vp]
    return L


def status_string(s: int) -> str:
    try:
        return lib().credit_status_string(int(s)).decode()
    except Exception:  # library not loadable: still give a readable message
        return f"status {s}"


def _check(st: int, what: str):
    if st != OK:
        raise CreditError(st, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def init(device: int | None = None):
    dev = torch.cuda.current_device() if device is None else int(device)
    _check(lib().credit_init(dev), "credit_init")


def _simple(fn_name, op, x, out, stream):
    if x.dim() != 2 or not x.is_contiguous():
        raise ValueError("expected a contiguous 2-D tensor")
    dt = DTYPE_OF[x.dtype]
    rows, cols = x.shape
    if out is None:
        out = torch.empty(rows, device=x.device, dtype=torch.float32) if op == LOGSUMEXP else torch.empty_like(x)
    _check(getattr(lib(), fn_name)(_ptr(x), _ptr(out), rows, cols, dt, _stream(stream)), fn_name)
    return out


def softmax(x, out=None, stream=None):
    return _simple("credit_softmax", SOFTMAX, x, out, stream)


def logsumexp(x, out=None, stream=None):
    return _simple("credit_logsumexp", LOGSUMEXP, x, out, stream)


def layernorm(x, out=None, stream=None):
    return _simple("credit_layernorm", LAYERNORM, x, out, stream)


def rmsnorm(x, out=None, stream=None):
    return _simple("credit_rmsnorm", RMSNORM, x, out, stream)


def make_plan(path: int, cluster_size: int = 1, ctas_per_row: int = 1, threads: int = 0, ring_chunks: int = 0,
              chunk_bytes: int = 0, reducer_threads: int = 0, retain: int = 0, fill_share: float = 0.0,
              fill_g: int = 0) -> PlanT:
    p = PlanT()
    p.path = path
    p.cluster_size = cluster_size
    p.ctas_per_row = ctas_per_row if path != PATH_CLUSTER else cluster_size
    p.threads = threads
    p.ring_chunks = ring_chunks
    p.chunk_bytes = chunk_bytes
    p.reducer_threads = reducer_threads
    p.retain = retain
    p.fill_share = fill_share
    p.fill_g = fill_g
    return p


def plan(op: int, rows: int, cols: int, in_dtype: int, out_dtype: int | None = None) -> PlanT:
    p = PlanT()
    if out_dtype is None:
        out_dtype = F32 if op == LOGSUMEXP else in_dtype
    _check(lib().credit_plan_ex(op, rows, cols, in_dtype, out_dtype, ctypes.byref(p)), "credit_plan_ex")
    return p


def make_args(op: int, x, out, *, rows: int | None = None, cols: int | None = None, in_dtype: int | None = None,
              out_dtype: int | None = None, ld_in: int = 0, ld_out: int = 0, in_scale=None, out_scale=None,
              gamma=None, beta=None, eps: float = -1.0) -> ArgsT:
    a = ArgsT()
    a.op = op
    a.in_ = _ptr(x)
    a.out = _ptr(out)
    if rows is None or cols is None:
        rows, cols = x.shape[0], x.shape[-1]
    a.rows, a.cols, a.ld_in, a.ld_out = rows, cols, ld_in, ld_out
    if in_dtype is None:
        in_dtype = DTYPE_OF[x.dtype]
    if out_dtype is None:
        out_dtype = F32 if op == LOGSUMEXP else (DTYPE_OF[out.dtype] if hasattr(out, "dtype") else in_dtype)
    a.in_dtype, a.out_dtype = in_dtype, out_dtype
    a.in_scale, a.out_scale = _ptr(in_scale), _ptr(out_scale)
    a.gamma, a.beta = _ptr(gamma), _ptr(beta)
    a.eps = eps
    return a


def plan_check(op: int, x, out, plan: PlanT, **kw) -> int:
    """credit_plan_check: OK if `plan` is legal for these arguments."""
    a = make_args(op, x, out, **kw)
    return lib().credit_plan_check(ctypes.byref(a), ctypes.byref(plan))


def max_clusters(op: int, x, out, plan: PlanT, **kw) -> int:
    """credit_max_clusters: co-resident clusters (CTAs for one-CTA) of a staged plan; 0 if illegal."""
    a = make_args(op, x, out, **kw)
    return int(lib().credit_max_clusters(ctypes.byref(a), ctypes.byref(plan)))


def run_ex(op: int, x, out, *, plan: PlanT | None = None, stream=None, **kw) -> int:
    """credit_run_ex.  x / out: tensors or raw device addresses; keyword
    arguments as make_args.  Returns the status (raises CreditError on a
    non-OK status)."""
    a = make_args(op, x, out, **kw)
    st = lib().credit_run_ex(ctypes.byref(a), ctypes.byref(plan) if plan is not None else None, _stream(stream))
    _check(st, "credit_run_ex")
    return st


def run_host(op: int, x, out, *, plan: PlanT | None = None, **kw) -> int:
    """credit_run_host: x / out (and in_scale, out_scale, gamma, beta) are
    host (CPU) tensors, pinned for full copy bandwidth; returns once out holds
    the result.  Raises CreditError on a non-OK status."""
    a = make_args(op, x, out, **kw)
    st = lib().credit_run_host(ctypes.byref(a), ctypes.byref(plan) if plan is not None else None)
    _check(st, "credit_run_host")
    return st


def run_two_pass_noalloc(op: int, x, out, ctas_per_row: int, *, stream=None, **kw) -> int:
    """credit_run_two_pass_noalloc: the split-row two-pass path with the
    library's fixed device scratch (no allocation).  Returns the status."""
    a = make_args(op, x, out, **kw)
    return lib().credit_run_two_pass_noalloc(ctypes.byref(a), int(ctas_per_row), _stream(stream))


def make_bwd_args(op: int, a, dy, dx, *, rows: int | None = None, cols: int | None = None, ld: int = 0,
                  dtype: int | None = None, gamma=None, mean=None, rstd=None, scale=None, dx2=None) -> BwdArgsT:
    r = BwdArgsT()
    r.op = op
    r.dtype = DTYPE_OF[a.dtype] if dtype is None else dtype
    r.a, r.dy, r.dx = _ptr(a), _ptr(dy), _ptr(dx)
    if rows is None or cols is None:
        rows, cols = a.shape[0], a.shape[-1]
    r.rows, r.cols, r.ld = rows, cols, ld
    r.gamma, r.mean, r.rstd, r.scale, r.dx2 = _ptr(gamma), _ptr(mean), _ptr(rstd), _ptr(scale), _ptr(dx2)
    return r


def run_bwd(op: int, a, dy, dx, *, plan: PlanT | None = None, stream=None, **kw) -> int:
    """credit_run_bwd: dx of softmax (a = y), LayerNorm or RMSNorm (a = x); keyword arguments as
    make_bwd_args (gamma, mean, rstd are FP32 tensors).  Raises CreditError on a non-OK status."""
    r = make_bwd_args(op, a, dy, dx, **kw)
    st = lib().credit_run_bwd(ctypes.byref(r), ctypes.byref(plan) if plan is not None else None, _stream(stream))
    _check(st, "credit_run_bwd")
    return st


def run_bwd_status(*args, **kw) -> int:
    try:
        return run_bwd(*args, **kw)
    except CreditError as e:
        return e.status


def plan_bwd(op: int, rows: int, cols: int, dtype: int) -> PlanT:
    p = PlanT()
    _check(lib().credit_plan_bwd(op, rows, cols, dtype, ctypes.byref(p)), "credit_plan_bwd")
    return p


def bwd_plan_check(op: int, a, dy, dx, plan: PlanT, **kw) -> int:
    r = make_bwd_args(op, a, dy, dx, **kw)
    return lib().credit_bwd_plan_check(ctypes.byref(r), ctypes.byref(plan))


def run_ex_status(*args, **kw) -> int:
    """Like run_ex but returns the status instead of raising."""
    try:
        return run_ex(*args, **kw)
    except CreditError as e:
        return e.status


def set_trace(buf=None) -> None:
    """credit_set_trace: buf is a uint64 CUDA tensor (or None to stop)."""
    if buf is None:
        _check(lib().credit_set_trace(None, 0), "credit_set_trace")
    else:
        _check(lib().credit_set_trace(_ptr(buf), buf.numel() * buf.element_size()), "credit_set_trace")


def microbench(runs: int = 15) -> dict:
    m = MicrobenchT()
    _check(lib().credit_microbench(ctypes.byref(m), runs), "credit_microbench")
    return m.as_dict()


def control_time(op: int, rows: int, cols: int, dtype: int, P: int, reps: int = 15) -> float:
    us = ctypes.c_float()
    _check(lib().credit_control_time(op, rows, cols, dtype, P, reps, ctypes.byref(us)), "credit_control_time")
    return us.value


def model_eval(**kw) -> dict:
    """credit_model_eval: the Eq. 7-9 terms for explicit inputs (host only)."""
    i = ModelInT()
    for k, v in kw.items():
        setattr(i, k, v)
    o = ModelOutT()
    _check(lib().credit_model_eval(ctypes.byref(i), ctypes.byref(o)), "credit_model_eval")
    return {k: getattr(o, k) for k in MODEL_OUT_FIELDS}


def calibrate(path: str, max_bytes: int = 0) -> None:
    _check(lib().credit_calibrate(path.encode(), max_bytes), "credit_calibrate")


def load_model(path: str) -> None:
    _check(lib().credit_load_model(path.encode()), "credit_load_model")


class Ragged:
    """credit_ragged_* handle: rows (in_off, out_off, cols, op) of one dtype."""

    def __init__(self, rows, dtype: int, in_base, out_base, tune: bool = True):
        arr = (RaggedRowT * len(rows))()
        for i, (io, oo, cols, op) in enumerate(rows):
            arr[i].in_off, arr[i].out_off, arr[i].cols, arr[i].op = int(io), int(oo), int(cols), int(op)
        h = ctypes.c_void_p()
        _check(lib().credit_ragged_create(arr, len(rows), dtype, _ptr(in_base), _ptr(out_base), int(tune),
                                          ctypes.byref(h)), "credit_ragged_create")
        self.h = h

    def run(self, stream=None):
        _check(lib().credit_ragged_run(self.h, _stream(stream)), "credit_ragged_run")

    def info(self) -> dict:
        i = RaggedInfoT()
        _check(lib().credit_ragged_info(self.h, ctypes.byref(i)), "credit_ragged_info")
        return {k: getattr(i, k) for k, _ in i._fields_}

    def close(self):
        if self.h:
            lib().credit_ragged_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_FEATURES = 21


def _fptr(a):
    import numpy as np
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mlp_num_params() -> int:
    return int(lib().credit_mlp_num_params())


def mlp_features(op, in_dtype, out_dtype, rows, cols, path, P, G, retain=0, fill_share=0.0):
    import numpy as np
    f = np.zeros(MLP_FEATURES, dtype=np.float32)
    _check(lib().credit_mlp_features(op, in_dtype, out_dtype, rows, cols, path, P, G, retain, float(fill_share),
                                     _fptr(f)),
           "credit_mlp_features")
    return f


def mlp_train(X, y, *, epochs=200, batch=256, lr=2e-3, seed=0):
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    curve = np.zeros(epochs, dtype=np.float32)
    _check(lib().credit_mlp_train(_fptr(X), _fptr(y), X.shape[0], epochs, batch, lr, seed, _fptr(curve)),
           "credit_mlp_train")
    return curve


def mlp_train_ensemble(X, y, *, members=5, epochs=200, batch=256, lr=2e-3, seed=0):
    """credit_mlp_train_ensemble: `members` networks (seeds seed, seed+1, ...),
    predictions averaged; returns the first member's loss curve."""
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    curve = np.zeros(epochs, dtype=np.float32)
    _check(lib().credit_mlp_train_ensemble(_fptr(X), _fptr(y), X.shape[0], members, epochs, batch, lr, seed,
                                           _fptr(curve)), "credit_mlp_train_ensemble")
    return curve


def mlp_members() -> int:
    return int(lib().credit_mlp_members())


def mlp_predict(X):
    import numpy as np
    X = np.ascontiguousarray(X, dtype=np.float32)
    out = np.zeros(X.shape[0], dtype=np.float32)
    _check(lib().credit_mlp_predict(_fptr(X), X.shape[0], _fptr(out)), "credit_mlp_predict")
    return out


def mlp_grad(params, X, t):
    import numpy as np
    params = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    t = np.ascontiguousarray(t, dtype=np.float32)
    g = np.zeros(mlp_num_params(), dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(lib().credit_mlp_grad(_fptr(params), _fptr(X), _fptr(t), X.shape[0], _fptr(g), _fptr(loss)),
           "credit_mlp_grad")
    return float(loss[0]), g


def mlp_adam_step(params, grad, m, v, step: int, lr: float):
    """One Adam step of the training kernel: returns the new (params, m, v)."""
    import numpy as np
    p = np.array(params, dtype=np.float32)
    mm = np.array(m, dtype=np.float32)
    vv = np.array(v, dtype=np.float32)
    g = np.ascontiguousarray(grad, dtype=np.float32)
    _check(lib().credit_mlp_adam_step(_fptr(p), _fptr(g), _fptr(mm), _fptr(vv), int(step), float(lr)),
           "credit_mlp_adam_step")
    return p, mm, vv


def mlp_save(path: str):
    _check(lib().credit_mlp_save(path.encode()), "credit_mlp_save")


def mlp_load(path: str):
    _check(lib().credit_mlp_load(path.encode()), "credit_mlp_load")


def dataflow(op: int, in_dtype: int = F32) -> DataflowT:
    """credit_dataflow_of: the structural description of an op the screen reads."""
    d = DataflowT()
    _check(lib().credit_dataflow_of(op, in_dtype, ctypes.byref(d)), "credit_dataflow_of")
    return d


def screen(d: DataflowT, P: int = 16):
    """credit_screen: (verdict, K) for cluster size P."""
    v, k = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().credit_screen(ctypes.byref(d), P, ctypes.byref(v), ctypes.byref(k)), "credit_screen")
    return v.value, k.value


def plan_control(op: int, rows: int, cols: int):
    """credit_plan_control: (plan, screen verdict) of a control op."""
    p, v = PlanT(), ctypes.c_int32()
    _check(lib().credit_plan_control(op, rows, cols, ctypes.byref(p), ctypes.byref(v)), "credit_plan_control")
    return p, v.value


def run_control(op: int, x, out, *, rows=None, cols=None, ld_in=0, ld_out=0, weights=None, stream=None) -> int:
    """credit_run_control: the scan / stencil control ops on FP32 device rows (weights: FP32 device tensor of
    2 r + 1 values for the stencil).  Raises CreditError on a non-OK status."""
    if rows is None or cols is None:
        rows, cols = x.shape[0], x.shape[-1]
    radius = 0 if weights is None else (weights.numel() - 1) // 2
    st = lib().credit_run_control(op, _ptr(x), _ptr(out), rows, cols, ld_in, ld_out, _ptr(weights), radius,
                                  _stream(stream))
    _check(st, "credit_run_control")
    return st


def run_control_status(*args, **kw) -> int:
    try:
        return run_control(*args, **kw)
    except CreditError as e:
        return e.status


def set_wait_test(wait_ns: int = 0, extra_tx_bytes: int = 0) -> None:
    """credit_set_wait_test (test only): short chunk-wait limit and an unsatisfiable first-chunk barrier."""
    _check(lib().credit_set_wait_test(int(wait_ns), int(extra_tx_bytes)), "credit_set_wait_test")


def device_error(stream=None) -> int:
    return lib().credit_device_error(_stream(stream))


def slice_capacity(dtype: int) -> int:
    return int(lib().credit_slice_capacity(dtype))


def launch_count() -> int:
    return int(lib().credit_launch_count())
