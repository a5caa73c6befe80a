"""CPU-side checks of the C ABI: the library builds, loads and exports every
entry point declared in include/*.h, and argument validation rejects bad
calls before anything touches a GPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_2609_01864_gb300 import build as B
from paper_2609_01864_gb300 import credit as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return C.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(credit_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("credit_softmax", "credit_logsumexp", "credit_layernorm", "credit_rmsnorm", "credit_plan",
              "credit_run_ex", "credit_init"):
        assert n in names


def test_every_declared_function_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    assert C.status_string(C.OK) == "CREDIT_OK"
    assert C.status_string(C.ERR_INVALID_ARG) == "CREDIT_ERR_INVALID_ARG"
    assert C.status_string(99) == "CREDIT_ERR_UNKNOWN"
    assert lib.credit_version() >= 10000


def test_validation_rejects_bad_calls_without_touching_the_gpu(lib):
    # NULL argument block
    assert lib.credit_run_ex(None, None, None) == C.ERR_INVALID_ARG
    a = C.ArgsT()
    a.op, a.in_, a.out, a.rows, a.cols = C.SOFTMAX, 0x1000, 0x2000, 4, 0   # cols == 0
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.cols, a.op = 16, 7                                                   # unknown op
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.op, a.in_dtype = C.SOFTMAX, C.FP8_E4M3                                # FP8 without scales
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.in_dtype, a.in_ = C.F32, 0x1002                                      # misaligned FP32 pointer
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.in_, a.op, a.out = 0x1000, C.LOGSUMEXP, 0x1000                       # in == out for logsumexp
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.op, a.out, a.in_ = C.SOFTMAX, 0x2000, None                            # NULL input
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG
    a.in_, a.rows = 0x1000, 0                                              # rows == 0 is a no-op
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.OK
    # int8 quantisation: codes only as its output, with scales, from FP32 / BF16 rows
    a.rows, a.op, a.in_dtype, a.out_dtype, a.out_scale = 4, C.QUANT_INT8, C.F32, C.F32, 0x3000
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG   # not an int8 output
    a.op, a.out_dtype = C.SOFTMAX, C.INT8
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG   # int8 output of another op
    a.op, a.out_scale = C.QUANT_INT8, None
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_INVALID_ARG   # no scales
    a.out_scale, a.in_dtype, a.in_scale = 0x3000, C.FP8_E4M3, 0x4000
    assert lib.credit_run_ex(ctypes.byref(a), None, None) == C.ERR_UNSUPPORTED   # FP8 rows
    a.in_dtype, a.out_dtype, a.out_scale, a.in_scale = C.F32, C.F32, None, None
    # the wait-test knob checks its arguments on the host
    assert lib.credit_set_wait_test(-1, 0) == C.ERR_INVALID_ARG
    assert lib.credit_set_wait_test(0, 8) == C.ERR_INVALID_ARG
    assert lib.credit_set_wait_test(0, 0) == C.OK
    # simple entry points: FP8 needs credit_run_ex (scales)
    assert lib.credit_softmax(0x1000, 0x2000, 4, 16, C.FP8_E4M3, None) == C.ERR_INVALID_ARG
    p = C.PlanT()
    assert lib.credit_plan_ex(9, 4, 16, 0, 0, ctypes.byref(p)) == C.ERR_INVALID_ARG
    assert lib.credit_plan_ex(0, 4, 0, 0, 0, ctypes.byref(p)) == C.ERR_INVALID_ARG
    assert lib.credit_plan_ex(0, 4, 16, 0, 0, None) == C.ERR_INVALID_ARG


def test_backward_validation_rejects_bad_calls_without_touching_the_gpu(lib):
    assert lib.credit_run_bwd(None, None, None) == C.ERR_INVALID_ARG
    r = C.BwdArgsT()
    r.op, r.dtype, r.a, r.dy, r.dx, r.rows, r.cols = C.SOFTMAX_BWD, C.F32, 0x1000, 0x2000, 0x3000, 4, 16
    for op in (C.RMSNORM, 9, -1):                                           # not a backward op
        r.op = op
        assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op, r.dtype = C.SOFTMAX_BWD, C.FP8_E4M3                               # FP8: no backward kernels
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_UNSUPPORTED
    r.dtype, r.ld = C.F32, 8                                                # ld < cols
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.ld, r.cols = 0, 0                                                     # cols == 0
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.cols, r.dx = 16, None                                                 # NULL output
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.dx, r.op = 0x3000, C.LAYERNORM_BWD                                    # LayerNorm needs mean and rstd
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.rstd = 0x4000
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op, r.rstd = C.RMSNORM_BWD, None                                       # RMSNorm needs rstd
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op, r.rstd = C.WVAR_BWD, None                                          # two-output ops need dx2
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op = C.PEARSON_BWD
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op = 11                                                               # past the last backward op
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.ERR_INVALID_ARG
    r.op, r.rows = C.RMSNORM_BWD, 0                                         # rows == 0 is a no-op
    assert lib.credit_run_bwd(ctypes.byref(r), None, None) == C.OK
    p = C.PlanT()
    assert lib.credit_plan_bwd(C.SOFTMAX, 4, 16, C.F32, ctypes.byref(p)) == C.ERR_INVALID_ARG
    assert lib.credit_plan_bwd(C.XENT_BWD, 4, 0, C.F32, ctypes.byref(p)) == C.ERR_INVALID_ARG
    assert lib.credit_plan_bwd(C.XENT_BWD, 4, 16, C.FP8_E4M3, ctypes.byref(p)) == C.ERR_UNSUPPORTED
    assert lib.credit_plan_bwd(C.XENT_BWD, 4, 16, C.F32, None) == C.ERR_INVALID_ARG


def test_struct_layouts_match_the_header():
    assert ctypes.sizeof(C.PlanT) == 56 and C.PlanT.smem_bytes.offset == 32 and C.PlanT.fill_g.offset == 52
    assert ctypes.sizeof(C.ArgsT) == 104
    assert C.ArgsT.eps.offset == 96 and C.ArgsT.in_scale.offset == 64


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """Every ctypes mirror of a header struct has the C compiler's size and field offsets."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    cuda_inc = "/usr/local/cuda/include"
    if cc is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime_api.h")):
        pytest.skip("no C compiler or CUDA headers")
    structs = {"credit_plan_t": C.PlanT, "credit_args": C.ArgsT, "credit_bwd_args": C.BwdArgsT}
    rename = {"in_": "in"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "credit.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {rename.get(f, f)}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-I", cuda_inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        cname, field, val = line.split()
        py = structs[cname]
        got = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert got == int(val), (cname, field, got, val)


def test_binding_constants_match_the_header_enums():
    """Every enum value the binding hard-codes is the header's."""
    text = open(os.path.join(ROOT, "include", "credit.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(CREDIT_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    expect = {
        "CREDIT_F32": C.F32, "CREDIT_BF16": C.BF16, "CREDIT_FP8_E4M3": C.FP8_E4M3,
        "CREDIT_OP_SOFTMAX": C.SOFTMAX, "CREDIT_OP_LOGSUMEXP": C.LOGSUMEXP, "CREDIT_OP_LAYERNORM": C.LAYERNORM,
        "CREDIT_OP_RMSNORM": C.RMSNORM, "CREDIT_PATH_AUTO": C.PATH_AUTO, "CREDIT_PATH_ONE_CTA": C.PATH_ONE_CTA,
        "CREDIT_PATH_TWO_PASS": C.PATH_TWO_PASS, "CREDIT_PATH_CLUSTER": C.PATH_CLUSTER,
        "CREDIT_RETAIN_AUTO": C.RETAIN_AUTO, "CREDIT_RETAIN_SMEM": C.RETAIN_SMEM, "CREDIT_RETAIN_TMEM": C.RETAIN_TMEM,
        "CREDIT_OK": C.OK, "CREDIT_ERR_INVALID_ARG": C.ERR_INVALID_ARG, "CREDIT_ERR_UNSUPPORTED": C.ERR_UNSUPPORTED,
        "CREDIT_ERR_CUDA": C.ERR_CUDA, "CREDIT_ERR_TIMEOUT": C.ERR_TIMEOUT,
        "CREDIT_ERR_NOT_INITIALIZED": C.ERR_NOT_INITIALIZED, "CREDIT_ERR_CAPTURE": C.ERR_CAPTURE,
        "CREDIT_ERR_IO": C.ERR_IO, "CREDIT_OP_SOFTMAX_BWD": C.SOFTMAX_BWD,
        "CREDIT_OP_LAYERNORM_BWD": C.LAYERNORM_BWD, "CREDIT_OP_RMSNORM_BWD": C.RMSNORM_BWD,
        "CREDIT_OP_SOFTMAX_LOGITS_BWD": C.SOFTMAX_LOGITS_BWD, "CREDIT_OP_XENT_BWD": C.XENT_BWD,
        "CREDIT_OP_WVAR_BWD": C.WVAR_BWD, "CREDIT_OP_PEARSON_BWD": C.PEARSON_BWD,
        "CREDIT_INT8": C.INT8, "CREDIT_OP_QUANT_INT8": C.QUANT_INT8,
    }
    for name, v in expect.items():
        assert vals.get(name) == v, (name, vals.get(name), v)
    assert C.MLP_FEATURES == int(re.search(r"#define CREDIT_MLP_FEATURES (\d+)", text).group(1))
