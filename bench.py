"""Benchmark of the reduction-reuse row ops on GB300 (one JSON line on stdout).

Workload (a "step"): LayerNorm (gamma ~ N(1, 0.1), beta ~ N(0, 0.1)) and
RMSNorm (gamma) in FP32 over 4096 rows x cols in {16K, 64K, 128K, 256K, 512K},
inputs N(0, 1) with 1% outliers at +-50, each shape run once through the
public C ABI with the plan the cost model picks.  Every input tensor (>= 268
MB) is larger than the 129 MB L2, so no flush is needed between steps.

value      algorithmic HBM GB/s of the whole step (one read of every input
           element, one write of every output element; gamma/beta excluded)
           with inputs resident in HBM, timed with CUDA events, max over ranks
e2e        the same metric end to end: pinned host inputs copied in, the ops
           run, the outputs copied back, all inside the timed region
roofline   the dominant kernel's achieved GB/s (its algorithmic bytes per
           launch / its mean launch time, CUDA events on the launching stream)
           against the measured HBM copy rate
cpu_baseline  the FP64 oracle on a bounded sample of the same shapes, all
           host cores

Also reported: speedup of the chosen plans over the best non-DSMEM plan
(one-CTA staging or two-pass reread) on the same shapes, and the cost model's
pick accuracy on these shapes (pick within 5% of the measured best candidate);
`backward`: the gradient ops (softmax, LayerNorm, RMSNorm, softmax from
logits, cross entropy, weighted variance, Pearson correlation) over 4096 rows
x {16K, 64K, 128K, 256K} FP32; `quant_int8`: row-wise int8 quantisation of
4096 x {16K, 64K, 256K} FP32 rows; `precision`: softmax and log-sum-exp over
4096 x {128K, 256K} BF16 / FP8-E4M3 logits N(0, 3^2) with the error of sampled
rows against the oracle; `ragged`: 20000 BF16 rows of log-uniform width in one
graph-replayed persistent launch; `controls`: the screen's negative controls
(row scan, row stencil) planned and timed on the global path.  In every table each candidate plan is
timed beside the planner's pick (outside the timed step).  `summary`, last on
the line, repeats each table's headline figures.

--impl reference  times the FP64 CPU oracle (the reference arm of this
           project) on a bounded sample of the same workload.
--case op:rows:cols:path:P  runs one small case a few times (for profilers; ops 4-10 are the
           backward ops, 11 the int8 quantisation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WIDTHS = [16384, 65536, 131072, 262144, 524288]
ROWS = 4096
OPS = ("layernorm", "rmsnorm")
METRIC = "HBM GB/s (% of roofline) & speedup vs best non-DSMEM path; cost-model pick accuracy"
FALLBACK_HBM_GBS = 6800.0


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def algorithmic_bytes(rows, cols, op):
    return rows * cols * 8  # FP32 in + FP32 out


def kernel_name(plan, C, cols=0, isz=4):
    if plan.path in (C.PATH_ONE_CTA, C.PATH_CLUSTER):
        if plan.path == C.PATH_CLUSTER and plan.fill_share > 0:
            return "k_ring_tm+fill" if plan.retain == C.RETAIN_TMEM else "k_ring+fill"
        if plan.retain == C.RETAIN_TMEM:
            return "k_ring_tm"
        if plan.retain == C.RETAIN_AUTO:  # the library's AUTO rule for the norms with FP32 output
            P = max(1, plan.cluster_size)
            body = -(-(cols * isz // 16) // P) * 16
            if 32768 < body <= 8 * 16384 and os.environ.get("CREDIT_RETAIN", "") != "smem":
                return "k_ring_tm"
        return "k_ring"
    return "k_tp_fused" if plan.ctas_per_row == 1 else "k_tp_split"


def source_sha():
    """Hash of the row-kernel sources a traffic capture was taken on."""
    h = hashlib.sha256()
    for name in ("credit_prim.cuh", "credit_rows.cuh", "credit_ring_tm.cuh"):
        with open(os.path.join(ROOT, "paper_2609_01864_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_record(kernel: str, op: str, cols: int):
    """Per-launch DRAM bytes from a committed ncu summary, if it was taken on
    the kernel source as it is now (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            recs = json.load(f)
    except Exception:
        return None
    h = source_sha()
    for r in recs.get("records", []):
        if r.get("kernel") == kernel and r.get("op") == op and r.get("cols") == cols and r.get("source_sha") == h:
            return r
    return None


def time_events(fn, reps, warm=1):
    import torch
    for _ in range(warm):
        fn()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def candidates(C, op, x, y, g=None, b=None, fills=True, **kw):
    """Every legal plan of one call: one-CTA / cluster P = 2..16 in both retention tiers, fills of cluster
    plans that leave SMs idle, two-pass G = 1, 2, 4, 8."""
    import torch
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    kw = dict(kw, gamma=g, beta=b)
    out = []
    for P in (1, 2, 4, 8, 16):
        legal = []
        for retain, tag in ((C.RETAIN_SMEM, ""), (C.RETAIN_TMEM, "_tm")):
            p = C.make_plan(C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER, P, retain=retain)
            if C.plan_check(op, x, y, p, **kw) == C.OK:
                name = f"{'one_cta' if P == 1 else 'cluster'}{'' if P == 1 else P}{tag}"
                out.append((name, p))
                legal.append((name, retain, p))
        if fills and P > 1 and legal:  # fills of a cluster plan that leaves SMs idle
            name, retain, p = legal[-1]
            if sm - P * C.max_clusters(op, x, y, p, **kw) >= 16:
                for f in (0.15, 0.2, 0.3, 0.4):
                    out.append((f"{name}_f{f}", C.make_plan(C.PATH_CLUSTER, P, retain=retain, fill_share=f)))
    for G in (1, 2, 4, 8):
        p = C.make_plan(C.PATH_TWO_PASS, ctas_per_row=G)
        out.append((f"two_pass_g{G}", p))
    return out


# ---------------------------------------------------------------- reference arm
def cpu_oracle_sample(seconds: float = 10.0, threads: int = 0):
    """Time the FP64 oracle on a bounded sample of the workload (rows of each
    shape, both ops), repeating until `seconds` have elapsed."""
    import numpy as np
    import oracle as O
    from paper_2609_01864_gb300 import synth
    O.build()
    rows_per = 8
    data = []
    for cols in WIDTHS:
        x = synth.outliers(rows_per, cols, seed=synth.SEED_DATA).numpy()
        g, bt = synth.gamma_beta(cols)
        data.append((cols, x, g.numpy(), bt.numpy()))
    nbytes = 0
    t0 = time.perf_counter()
    reps = 0
    while True:
        for cols, x, g, bt in data:
            for op in (O.LAYERNORM, O.RMSNORM):
                O.run(op, O.F32, x, rows_per, cols, gamma=g, beta=bt if op == O.LAYERNORM else None,
                      want_exact=False, want_encoded=True, nthreads=threads)
                nbytes += rows_per * cols * 8
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    cores = threads if threads > 0 else O.max_threads()
    return {"value": round(nbytes / el / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{rows_per} rows x each of cols {WIDTHS}, LayerNorm+RMSNorm, FP32 in/out, "
                      f"{reps} repetitions in {el:.1f} s ({nbytes / 1e9:.2f} GB algorithmic)"}


# ---------------------------------------------------------------- ranks (host logic, also run under gloo in tests)
def dist_env():
    """(rank, world, local rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest of the ranks' values (the step time the job is charged)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def ragged_shard(widths, world: int, rank: int):
    """Rows [lo, hi) of this rank's share of a ragged batch: the row list is cut where the running element
    count crosses k / world of the total (byte-balanced prefix sums; every share is contiguous and the shares
    differ by less than one row's bytes)."""
    import numpy as np
    ends = np.cumsum(np.asarray(widths, dtype=np.int64))
    total = int(ends[-1]) if len(ends) else 0

    def cut(k):
        if k <= 0:
            return 0
        if k >= world:
            return len(ends)
        return int(np.searchsorted(ends, total * k / world, side="right"))
    return cut(rank), cut(rank + 1)


def job_value(step_bytes_per_rank: int, world: int, ms_step: float) -> float:
    """Whole-job GB/s: every rank processes its own rows (weak scaling)."""
    return step_bytes_per_rank * world / (ms_step * 1e-3) / 1e9


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    per_step = min(10.0, max(0.05, args.ref_seconds / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_sample(seconds=min(2.0, per_step))
    vals = []
    last = None
    t0 = time.perf_counter()
    for _ in range(args.steps):
        last = cpu_oracle_sample(seconds=per_step)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {"metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el * 1e3 / max(1, args.steps), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "LayerNorm+RMSNorm FP32, 4096 x {16K,64K,128K,256K,512K} (bounded CPU sample)"},
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": last["cores"], "kind": "oracle",
                             "sample": last["sample"]},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_case(spec: str):
    import torch
    from paper_2609_01864_gb300 import build as B
    from paper_2609_01864_gb300 import credit as C
    from paper_2609_01864_gb300 import synth
    B.build()
    v = spec.split(":")
    op, rows, cols, path, P = [int(t) for t in v[:5]]
    retain = int(v[5]) if len(v) > 5 else 0
    fill = float(v[6]) if len(v) > 6 else 0.0
    C.init(torch.cuda.current_device())
    if C.SOFTMAX_BWD <= op <= C.PEARSON_BWD:  # backward op: a, dy -> dx (and dx2)
        a = synth.outliers(rows, cols, seed=synth.SEED_DATA, device="cuda")
        dy = synth.normal(rows, cols, seed=synth.SEED_DATA + 1, device="cuda")
        dx = torch.empty_like(a)
        g, _ = synth.gamma_beta(cols, device="cuda")
        st = torch.ones(rows, device="cuda")
        if op in (C.WVAR_BWD, C.PEARSON_BWD):
            if op == C.WVAR_BWD:
                dy = dy.abs() + 0.1  # weights
            kw = dict(scale=st, dx2=torch.empty_like(a))
        elif op in (C.LAYERNORM_BWD, C.RMSNORM_BWD):
            kw = dict(gamma=g, rstd=st, mean=st if op == C.LAYERNORM_BWD else None)
        else:
            kw = {}
        plan = None if path < 0 else C.make_plan(path, P, ctas_per_row=P if path == C.PATH_TWO_PASS else 1)
        for _ in range(3):
            C.run_bwd(op, a, dy, dx, plan=plan, **kw)
        torch.cuda.synchronize()
        assert C.device_error() == C.OK
        print(json.dumps({"case": spec, "launches": C.launch_count()}))
        return 0
    dtype = v[7] if len(v) > 7 else "f32"
    x = synth.outliers(rows, cols, seed=synth.SEED_DATA, device="cuda")
    g, b = synth.gamma_beta(cols, device="cuda")
    plan = None if path < 0 else C.make_plan(path, P, ctas_per_row=P if path == C.PATH_TWO_PASS else 1,
                                             retain=retain, fill_share=fill)
    if dtype == "e4m3":  # config-3 logits N(0, 3^2) as per-row scaled E4M3 codes
        x, isc = synth.to_e4m3_rowscaled(3.0 * synth.normal(rows, cols, seed=synth.SEED_DATA, device="cuda"))
        if op == C.LOGSUMEXP:
            y = torch.empty(rows, device="cuda")
            kw = dict(in_scale=isc)
        else:
            y = torch.empty_like(x)
            kw = dict(in_scale=isc, out_dtype=C.FP8_E4M3, out_scale=torch.empty(rows, device="cuda"))
    elif dtype == "bf16":
        x = x.to(torch.bfloat16)
        y = torch.empty(rows, device="cuda") if op == C.LOGSUMEXP else torch.empty_like(x)
        kw = {}
    elif op == C.QUANT_INT8:
        y = torch.empty(rows, cols, dtype=torch.int8, device="cuda")
        kw = dict(out_dtype=C.INT8, out_scale=torch.empty(rows, device="cuda"))
    else:
        y = torch.empty_like(x)
        kw = dict(gamma=g if op in (C.LAYERNORM, C.RMSNORM) else None, beta=b if op == C.LAYERNORM else None)
    for _ in range(3):
        C.run_ex(op, x, y, plan=plan, **kw)
    torch.cuda.synchronize()
    assert C.device_error() == C.OK
    print(json.dumps({"case": spec, "launches": C.launch_count()}))
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2609_01864_gb300 import build as B
    from paper_2609_01864_gb300 import credit as C
    from paper_2609_01864_gb300 import synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    C.init(local)
    calib = os.path.join(ROOT, "paper_2609_01864_gb300", "data", "gb300.calib")
    if os.path.exists(calib) and not args.no_model:
        C.load_model(calib)
    dev = torch.device("cuda", local)
    widths = WIDTHS if not args.widths else [int(w) for w in args.widths.split(",")]

    # ---- inputs (seeded, resident in HBM)
    shapes = []
    for cols in widths:
        x = synth.outliers(ROWS, cols, seed=synth.SEED_DATA + rank, device=dev)
        g, b = synth.gamma_beta(cols, device=dev)
        shapes.append({"cols": cols, "x": x, "y": torch.empty_like(x), "g": g, "b": b})
    jobs = []
    for sh in shapes:
        for name in OPS:
            op = C.LAYERNORM if name == "layernorm" else C.RMSNORM
            plan = C.plan(op, ROWS, sh["cols"], C.F32)
            kw = dict(gamma=sh["g"], beta=sh["b"] if op == C.LAYERNORM else None)
            jobs.append({"op": op, "name": name, "cols": sh["cols"], "x": sh["x"], "y": sh["y"], "kw": kw,
                         "plan": plan, "kernel": kernel_name(plan, C, sh["cols"]),
                         "bytes": algorithmic_bytes(ROWS, sh["cols"], op)})
    step_bytes = sum(j["bytes"] for j in jobs)
    stream = torch.cuda.current_stream()

    def step(record=None):
        for k, j in enumerate(jobs):
            if record is not None:
                record[k][0].record(stream)
            C.run_ex(j["op"], j["x"], j["y"], plan=j["plan"], **j["kw"])
            if record is not None:
                record[k][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    per = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in jobs]
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    n0 = C.launch_count()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(per[s])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = C.launch_count() - n0
    clk = clocks.stop()
    ms_total = max_over_ranks(t_start.elapsed_time(t_end), world, device=dev)
    ms_step = ms_total / args.steps
    value = job_value(step_bytes, world, ms_step)
    assert C.device_error() == C.OK

    # ---- per-kernel launch times (roofline of the dominant kernel)
    per_kernel = {}
    for s in range(args.steps):
        for k, j in enumerate(jobs):
            ms = per[s][k][0].elapsed_time(per[s][k][1])
            d = per_kernel.setdefault(j["kernel"], {"ms": 0.0, "launches": 0, "bytes": 0, "jobs": {}})
            d["ms"] += ms
            d["launches"] += 1
            d["bytes"] += j["bytes"]
            jd = d["jobs"].setdefault((j["name"], j["cols"]), {"ms": [], "bytes": j["bytes"]})
            jd["ms"].append(ms)
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dk = per_kernel[dom]
    peak, peak_kind = measured_peak()
    achieved = dk["bytes"] / (dk["ms"] * 1e-3) / 1e9
    # traffic of the dominant kernel's largest job (per launch), if a current capture exists
    big = max(dk["jobs"], key=lambda k: dk["jobs"][k]["bytes"])
    tr = traffic_record(dom, big[0], big[1])
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None if tr is None else tr["dram_bytes"],
                "peak_source": f"{peak_kind} hbm_gbs (copy)", "kernel": dom,
                "kernel_share": round(dk["ms"] / sum(v["ms"] for v in per_kernel.values()), 3),
                "traffic_job": None if tr is None else f"{big[0]} cols={big[1]}",
                "traffic_algorithmic_bytes": None if tr is None else tr.get("algorithmic_bytes")}
    per_job = []
    for k, j in enumerate(jobs):
        ms = statistics.median(per[s][k][0].elapsed_time(per[s][k][1]) for s in range(args.steps))
        per_job.append({"op": j["name"], "cols": j["cols"], "plan": C.PATH_NAMES[j["plan"].path],
                        "P": j["plan"].cluster_size, "G": j["plan"].ctas_per_row, "source": j["plan"].source,
                        "kernel": j["kernel"], "fill_share": round(j["plan"].fill_share, 3),
                        "ms": round(ms, 4), "GBps": round(j["bytes"] / ms / 1e6, 1)})

    # ---- end to end through the public API with host buffers (right after the
    # timed region, before the candidate sweep below)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(C, torch, dev, jobs, shapes, stream, args, world)

    # ---- speedup vs best non-DSMEM path and pick accuracy (every candidate timed)
    speed_num = speed_den = 0.0
    hits = 0
    pick_rows = []
    if not args.no_picks and world == 1:  # candidate tables time one GPU's kernels
        for k, j in enumerate(jobs):
            times = {}
            for name, p in candidates(C, j["op"], j["x"], j["y"], j["kw"]["gamma"], j["kw"]["beta"]):
                ts = time_events(lambda: C.run_ex(j["op"], j["x"], j["y"], plan=p, **j["kw"]), 5)
                times[name] = statistics.median(ts)
            best_non = min(v for n, v in times.items() if not n.startswith("cluster"))
            best_all = min(times.values())
            chosen = per_job[k]["ms"]
            speed_num += best_non
            speed_den += chosen
            hit = chosen <= 1.05 * best_all
            hits += int(hit)
            # paper-style profitability pair: the analytic model (Eq. 7-9, shared-memory staging) picks the
            # cluster path iff its best dT > 0; measured: best shared-memory cluster vs best non-DSMEM plan
            os.environ["CREDIT_MODEL"] = "analytic"
            ap_ = C.plan(j["op"], ROWS, j["cols"], C.F32)
            os.environ.pop("CREDIT_MODEL", None)
            cl = [v for n, v in times.items() if n.startswith("cluster") and not n.endswith("_tm")]
            pick_rows.append({"op": j["name"], "cols": j["cols"], "chosen_ms": chosen,
                              "best": min(times, key=times.get), "best_ms": round(best_all, 4),
                              "best_non_dsmem_ms": round(best_non, 4), "hit": hit,
                              "analytic_cluster": ap_.path == C.PATH_CLUSTER,
                              "measured_cluster": bool(cl) and min(cl) < best_non,
                              "candidates": {n: round(v, 4) for n, v in times.items()}})

    # the secondary tables time one GPU's kernels: at N = 1 only; the ragged batch is sharded across ranks
    single = world == 1
    bwd = None
    if not args.no_bwd and single:
        bwd = run_bwd_bench(C, torch, dev, synth)
    quant = run_quant_bench(C, torch, dev, synth) if not args.no_quant and single else None
    prec = run_precision_bench(C, torch, dev, synth) if not args.no_prec and single else None
    ragged = run_ragged_bench(C, torch, dev, synth, world=world, rank=rank) if not args.no_ragged else None
    controls = run_controls_bench(C, torch, dev, synth) if not args.no_controls and single else None

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_sample(seconds=args.cpu_seconds)

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "LayerNorm(gamma,beta)+RMSNorm(gamma) FP32, 4096 rows x cols "
                               "{16K,64K,128K,256K,512K}, N(0,1) with 1% +-50 outliers, planner-chosen path",
                   "rows": ROWS, "cols": widths, "ops": list(OPS),
                   "l2": "every input > L2 (>= 268 MB), no flush", "parallelism": f"rows per GPU x {world}"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "speedup_vs_best_non_dsmem": round(speed_num / speed_den, 4) if speed_den else None,
        "pick_accuracy": round(hits / len(jobs), 4) if pick_rows else None,
        "profitability": profitability(pick_rows) if pick_rows else None,
        "pick_rule": "chosen plan within 5% of the fastest measured candidate (median of 5)",
        "per_job": per_job,
        "picks": pick_rows,
        "backward": bwd,
        "quant_int8": quant,
        "precision": prec,
        "ragged": ragged,
        "controls": controls,
    }
    # the headline figures of every table, last on the line
    line["summary"] = {
        "forward": {"GBps": round(value, 1), "frac": round(value / roofline["peak"], 4),
                    "dominant_kernel_frac": roofline["frac"],
                    "speedup_vs_best_non_dsmem": line["speedup_vs_best_non_dsmem"],
                    "pick_accuracy": line["pick_accuracy"],
                    "per_job_GBps": {f"{j['op']}_{j['cols']}": j["GBps"] for j in per_job}},
        "backward": None if bwd is None else {k: bwd[k] for k in ("GBps", "speedup_vs_best_non_dsmem",
                                                                   "pick_accuracy")},
        "quant_int8": None if quant is None else {k: quant[k] for k in ("GBps", "speedup_vs_best_non_dsmem",
                                                                         "pick_accuracy", "sampled_rows_bit_exact")},
        "precision": None if prec is None else {
            "GBps": prec["GBps"], "max_err_in_bound_units": prec["max_err_in_bound_units"],
            "per_shape_GBps": {f"{r['op']}_{r['cols']}": r["chosen_GBps"] for r in prec["shapes"]}},
        "ragged": None if ragged is None else {k: ragged[k] for k in ("GBps", "frac", "ms", "max_err_in_bound_units")},
        "controls": None if controls is None else {
            "screen": controls["screen"], "GBps": {f"{r['op']}_{r['cols']}": r["GBps"] for r in controls["shapes"]}},
        "e2e_frac_of_link": None if e2e is None else e2e["frac_of_link_both"]}
    print(json.dumps(line), flush=True)
    return 0


BWD_WIDTHS = [16384, 65536, 131072, 262144]


def run_bwd_bench(C, torch, dev, synth):
    """The backward ops (dx of softmax, LayerNorm, RMSNorm; dz of softmax and of the cross entropy from
    logits, with the same arrays as logits and as targets; the two gradients of the weighted variance and of
    the Pearson correlation of a row pair; FP32, 4096 rows): every candidate plan timed (median of 5, CUDA
    events), the planner's pick, the best non-DSMEM plan and the speed-up of the pick over it.  Algorithmic
    bytes: one read of each input array and one write of each output (12 B per element, 16 for the pair
    ops)."""
    peak, peak_kind = measured_peak()
    out = {"rows": ROWS, "dtype": "f32", "peak_GBps": peak, "peak_source": peak_kind, "shapes": []}
    for cols in BWD_WIDTHS:
        a = synth.outliers(ROWS, cols, seed=synth.SEED_DATA, device=dev)
        dy = synth.normal(ROWS, cols, seed=synth.SEED_DATA + 1, device=dev)
        dx = torch.empty_like(a)
        g, _ = synth.gamma_beta(cols, device=dev)
        a64 = a.double()
        mean = a64.mean(dim=1)
        rstd_ln = (1.0 / torch.sqrt(((a64 - mean[:, None]) ** 2).mean(dim=1) + 1e-5)).float()
        rstd_rms = (1.0 / torch.sqrt((a64 * a64).mean(dim=1) + 1e-6)).float()
        mean = mean.float()
        del a64
        # the pair ops (f3): weighted variance of 2 a + 3 with weights U(0.1, 2); Pearson of a and 0.5 a + dy
        gen = torch.Generator(device=dev).manual_seed(synth.SEED_DATA + 7)
        wv_x = 2.0 * a + 3.0
        wv_w = 0.1 + 1.9 * torch.rand(ROWS, cols, generator=gen, device=dev)
        pe_y = 0.5 * a + dy
        g_row = 0.5 + 1.5 * torch.rand(ROWS, generator=gen, device=dev)
        dx2 = torch.empty_like(a)
        ops = ((C.SOFTMAX_BWD, "softmax_bwd", a, dy, {}),
               (C.LAYERNORM_BWD, "layernorm_bwd", a, dy, dict(gamma=g, mean=mean, rstd=rstd_ln)),
               (C.RMSNORM_BWD, "rmsnorm_bwd", a, dy, dict(gamma=g, rstd=rstd_rms)),
               (C.SOFTMAX_LOGITS_BWD, "softmax_logits_bwd", a, dy, {}),
               (C.XENT_BWD, "xent_bwd", a, dy, {}),
               (C.WVAR_BWD, "wvar_bwd", wv_x, wv_w, dict(scale=g_row, dx2=dx2)),
               (C.PEARSON_BWD, "pearson_bwd", a, pe_y, dict(scale=g_row, dx2=dx2)))
        for op, name, a_, dy_, kw in ops:
            nbytes = ROWS * cols * (16 if op in (C.WVAR_BWD, C.PEARSON_BWD) else 12)
            cands = [(f"two_pass_g{G}", C.make_plan(C.PATH_TWO_PASS, ctas_per_row=G)) for G in (1, 2, 4, 8)]
            cands.append(("one_cta", C.make_plan(C.PATH_ONE_CTA)))
            cands += [(f"cluster{P}", C.make_plan(C.PATH_CLUSTER, P)) for P in (2, 4, 8, 16)]
            times = {}
            for cname, p in cands:
                if C.bwd_plan_check(op, a_, dy_, dx, p, **kw) != C.OK:
                    continue
                ts = time_events(lambda: C.run_bwd(op, a_, dy_, dx, plan=p, **kw), 5)
                times[cname] = statistics.median(ts)
            chosen_plan = C.plan_bwd(op, ROWS, cols, C.F32)
            chosen = statistics.median(time_events(lambda: C.run_bwd(op, a_, dy_, dx, **kw), 5))
            non = {k: v for k, v in times.items() if k.startswith("two_pass")}
            staged = {k: v for k, v in times.items() if not k.startswith("two_pass")}
            best_non = min(non.values())
            pname = (PATH_NAMES_SHORT[chosen_plan.path] +
                     (str(chosen_plan.cluster_size) if chosen_plan.path == C.PATH_CLUSTER else
                      (f"_g{chosen_plan.ctas_per_row}" if chosen_plan.path == C.PATH_TWO_PASS else "")))
            out["shapes"].append({
                "op": name, "cols": cols, "bytes_per_elem": nbytes // (ROWS * cols), "chosen": pname,
                "chosen_ms": round(chosen, 4),
                "chosen_GBps": round(nbytes / chosen / 1e6, 1), "frac": round(nbytes / chosen / 1e6 / peak, 4),
                "best": min(times, key=times.get), "best_ms": round(min(times.values()), 4),
                "best_non_dsmem_ms": round(best_non, 4),
                "best_staged_ms": round(min(staged.values()), 4) if staged else None,
                "speedup_vs_best_non_dsmem": round(best_non / chosen, 4),
                "hit": chosen <= 1.05 * min(times.values()),
                "candidates": {k: round(v, 4) for k, v in sorted(times.items(), key=lambda kv: kv[1])}})
        del a, dy, dx, dx2, wv_x, wv_w, pe_y
        torch.cuda.empty_cache()
    assert C.device_error() == C.OK
    sh = out["shapes"]
    tot_chosen = sum(r["chosen_ms"] for r in sh)
    out["GBps"] = round(sum(ROWS * r["cols"] * r["bytes_per_elem"] for r in sh) / tot_chosen / 1e6, 1)
    out["speedup_vs_best_non_dsmem"] = round(sum(r["best_non_dsmem_ms"] for r in sh) / tot_chosen, 4)
    out["pick_accuracy"] = round(sum(r["hit"] for r in sh) / len(sh), 4)
    return out


def plan_name(C, p):
    """Short name of a plan, as the candidate tables spell it."""
    if p.path == C.PATH_TWO_PASS:
        return f"two_pass_g{p.ctas_per_row}"
    base = "one_cta" if p.path == C.PATH_ONE_CTA else f"cluster{p.cluster_size}"
    tag = "_tm" if p.retain == C.RETAIN_TMEM else ""
    return base + tag + (f"_f{round(p.fill_share, 2)}" if p.fill_share > 0 else "")


def time_candidates(C, op, x, y, kw, fills=False):
    """Median of 5 (CUDA events) for every legal plan of one call, and for the planner's own choice."""
    times = {}
    for name, p in candidates(C, op, x, y, fills=fills, **kw):
        times[name] = statistics.median(time_events(lambda: C.run_ex(op, x, y, plan=p, **kw), 5))
    chosen = statistics.median(time_events(lambda: C.run_ex(op, x, y, **kw), 5))
    return times, chosen


def table_row(name, cols, nbytes, times, chosen, chosen_name, peak):
    non = {k: v for k, v in times.items() if k.startswith("two_pass") or k.startswith("one_cta")}
    best = min(times.values())
    return {"op": name, "cols": cols, "chosen": chosen_name, "chosen_ms": round(chosen, 4),
            "chosen_GBps": round(nbytes / chosen / 1e6, 1), "frac": round(nbytes / chosen / 1e6 / peak, 4),
            "best": min(times, key=times.get), "best_ms": round(best, 4),
            "best_non_dsmem_ms": round(min(non.values()), 4),
            "speedup_vs_best_non_dsmem": round(min(non.values()) / chosen, 4), "hit": chosen <= 1.05 * best,
            "candidates": {k: round(v, 4) for k, v in sorted(times.items(), key=lambda kv: kv[1])[:6]}}


def table_summary(rows, nbytes_of):
    tot = sum(r["chosen_ms"] for r in rows)
    return {"GBps": round(sum(nbytes_of(r) for r in rows) / tot / 1e6, 1),
            "speedup_vs_best_non_dsmem": round(sum(r["best_non_dsmem_ms"] for r in rows) / tot, 4),
            "pick_accuracy": round(sum(r["hit"] for r in rows) / len(rows), 4)}


QUANT_WIDTHS = [16384, 65536, 262144]


def run_quant_bench(C, torch, dev, synth):
    """Row-wise int8 quantisation (the paper's suite, Sec. IV-A): FP32 rows of config 2's distribution,
    4096 x {16K, 64K, 256K}; every candidate timed beside the planner's pick; algorithmic bytes 4 in + 1 out
    per element + 4 per row (the scale).  Codes and scales of sampled rows are checked bit for bit against
    the oracle."""
    import numpy as np
    import oracle as O
    peak, peak_kind = measured_peak()
    out = {"rows": ROWS, "in_dtype": "f32", "bytes_per_elem": 5, "peak_GBps": peak, "peak_source": peak_kind,
           "shapes": []}
    exact = True
    for cols in QUANT_WIDTHS:
        x = synth.outliers(ROWS, cols, seed=synth.SEED_DATA, device=dev)
        q = torch.empty(ROWS, cols, dtype=torch.int8, device=dev)
        sc = torch.empty(ROWS, device=dev)
        kw = dict(out_dtype=C.INT8, out_scale=sc)
        times, chosen = time_candidates(C, C.QUANT_INT8, x, q, kw)
        nbytes = ROWS * cols * 5 + ROWS * 4
        pick = list(range(0, ROWS, ROWS // 8))
        qr, sr = O.quant_int8(x[pick].cpu().numpy())
        exact = exact and bool(np.array_equal(q[pick].cpu().numpy(), qr) and np.array_equal(sc[pick].cpu().numpy(), sr))
        out["shapes"].append(table_row("quant_int8", cols, nbytes, times, chosen,
                                       plan_name(C, C.plan(C.QUANT_INT8, ROWS, cols, C.F32, C.INT8)), peak))
        del x, q
        torch.cuda.empty_cache()
    assert C.device_error() == C.OK
    out.update(table_summary(out["shapes"], lambda r: ROWS * r["cols"] * 5 + ROWS * 4))
    out["sampled_rows_bit_exact"] = exact
    return out


PREC_WIDTHS = [131072, 262144]


def output_error(op, out_dt, y, ref, osc=None):
    """Largest error of sampled outputs in units of the output format's bound: FP32 (logsumexp) |y - y*| /
    max(|y*|, 1) / 1e-5; BF16 |y - y*| / ulp_bf16(y*); E4M3 |q s - y*| / (one E4M3 quantum at y* / s) s."""
    import numpy as np
    a = np.abs(ref)
    if out_dt == 0:
        return float(np.max(np.abs(y - ref) / np.maximum(a, 1.0)) / 1e-5)
    if out_dt == 1:
        e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
        ulp = np.where(a >= 2.0 ** -126, np.exp2(e - 7), 2.0 ** -133)
        return float(np.max(np.abs(y - ref) / ulp))
    s = np.asarray(osc, dtype=np.float64).reshape(-1, 1)
    t = a / s
    e = np.floor(np.log2(np.where(t > 0, t, 2.0 ** -30)))
    return float(np.max(np.abs(y * s - ref) / (np.exp2(np.maximum(e, -6) - 3) * s)))


def run_precision_bench(C, torch, dev, synth):
    """The precision workload: softmax and log-sum-exp over 4096 x {128K, 256K} logits N(0, 3^2) in BF16 and
    in FP8-E4M3 with a per-row FP32 scale, FP32 accumulation.  Every candidate timed beside the planner's
    pick; algorithmic bytes one read and one write (softmax BF16 4 B, FP8 2 B per element + 8 B per row;
    log-sum-exp BF16 2 B, FP8 1 B per element + 4 or 8 B per row).  Error of 8 sampled rows against the FP64
    oracle in units of each format's bound (<= 1 passes)."""
    import numpy as np
    import oracle as O
    peak, peak_kind = measured_peak()
    out = {"rows": ROWS, "logits": "N(0, 3^2)", "peak_GBps": peak, "peak_source": peak_kind, "shapes": []}
    nb = {}
    for cols in PREC_WIDTHS:
        x32 = synth.normal(ROWS, cols, std=3.0, seed=synth.SEED_DATA, device=dev)
        for dt, dname in ((C.BF16, "bf16"), (C.FP8_E4M3, "fp8")):
            if dt == C.BF16:
                x, isc = synth.to_bf16(x32), None
            else:
                x, isc = synth.to_e4m3_rowscaled(x32)
            pick = list(range(0, ROWS, ROWS // 8))
            raw = x[pick].cpu().contiguous()
            raw = raw.view(torch.int16).numpy().view(np.uint16) if dt == C.BF16 else raw.view(torch.uint8).numpy()
            for op, oname in ((C.SOFTMAX, "softmax"), (C.LOGSUMEXP, "logsumexp")):
                if op == C.LOGSUMEXP:
                    y = torch.empty(ROWS, device=dev)
                    osc = None
                    out_dt = C.F32
                else:
                    y = torch.empty(ROWS, cols, dtype=x.dtype, device=dev)
                    osc = torch.empty(ROWS, device=dev) if dt == C.FP8_E4M3 else None
                    out_dt = dt
                kw = dict(in_dtype=dt, out_dtype=out_dt, in_scale=isc, out_scale=osc)
                times, chosen = time_candidates(C, op, x, y, kw)
                isz = 2 if dt == C.BF16 else 1
                per_row = (4 if op == C.LOGSUMEXP else 0) + (4 if dt == C.FP8_E4M3 else 0) + \
                    (4 if dt == C.FP8_E4M3 and op == C.SOFTMAX else 0)  # LSE out; FP8 in / out scales
                nbytes = ROWS * cols * (isz if op == C.LOGSUMEXP else 2 * isz) + ROWS * per_row
                ref, _, _ = O.run(op, dt, raw, len(pick), cols, in_scale=None if isc is None else isc[pick].cpu().numpy())
                yv = y[pick].double().cpu().numpy() if op == C.LOGSUMEXP else y[pick].float().double().cpu().numpy()
                err = output_error(op, out_dt, yv, ref, None if osc is None else osc[pick].cpu().numpy())
                p = C.plan(op, ROWS, cols, dt, out_dt)
                row = table_row(f"{oname}_{dname}", cols, nbytes, times, chosen, plan_name(C, p), peak)
                row["max_err_in_bound_units"] = round(err, 4)
                out["shapes"].append(row)
                nb[(row["op"], cols)] = nbytes
                del y
            del x
        del x32
        torch.cuda.empty_cache()
    assert C.device_error() == C.OK
    out.update(table_summary(out["shapes"], lambda r: nb[(r["op"], r["cols"])]))
    out["max_err_in_bound_units"] = {d: max(r["max_err_in_bound_units"] for r in out["shapes"] if r["op"].endswith(d))
                                     for d in ("bf16", "fp8")}
    return out


def run_ragged_bench(C, torch, dev, synth, reps=10, world=1, rank=0):
    """The batching workload: 20000 BF16 rows of widths round(2^(10 + 10 u)) (log-uniform in [1K, 1M]),
    softmax or RMSNorm by a fair coin per row, packed with no alignment padding, run as one persistent launch
    replayed from a CUDA graph (the library's autotuner picks cluster size, staging, threads and vector
    width).  GB/s at 4 B per element (one BF16 read, one BF16 write); 16 sampled rows checked against the
    FP64 oracle.  Under several ranks each runs its byte-balanced contiguous share of the rows
    (ragged_shard) and the batch time is the slowest rank's."""
    import numpy as np
    import oracle as O
    peak, peak_kind = measured_peak()
    widths_all, ops_all = synth.ragged_widths(20000)
    widths_all, ops_all = widths_all.numpy(), ops_all.numpy()
    lo, hi = ragged_shard(widths_all, world, rank)
    widths, ops = widths_all[lo:hi], ops_all[lo:hi]
    offs = np.concatenate([[0], np.cumsum(widths)[:-1]]).astype(np.int64)
    total = int(widths.sum())
    g = torch.Generator(device=dev).manual_seed(synth.SEED_RAGGED + rank)
    d_in = (torch.randn(total, generator=g, device=dev) * 2.0).to(torch.bfloat16)
    d_out = torch.empty_like(d_in)
    rows = [(int(o), int(o), int(w), int(op)) for o, w, op in zip(offs, widths, ops)]
    t0 = time.perf_counter()
    R = C.Ragged(rows, C.BF16, d_in, d_out, tune=True)
    t_create = time.perf_counter() - t0
    ms = statistics.median(time_events(lambda: R.run(), reps, warm=3))
    if world > 1:
        ms = max_over_ranks(ms, world, device=dev)
    info = R.info()
    worst = 0.0
    for i in np.linspace(0, len(rows) - 1, 16).astype(int):
        o, w, op = int(offs[i]), int(widths[i]), int(ops[i])
        raw = d_in[o:o + w].cpu().view(torch.int16).numpy().view(np.uint16)
        ref, _, _ = O.run(op, C.BF16, raw, 1, w)
        worst = max(worst, output_error(op, C.BF16, d_out[o:o + w].float().double().cpu().numpy().reshape(1, w), ref))
    assert C.device_error() == C.OK
    total = int(widths_all.sum())  # the whole batch, over all ranks
    nbytes = total * 4
    res = {"rows": len(widths_all), "elements": total, "dtype": "bf16", "ms": round(ms, 4), "ranks": world,
           "GBps": round(nbytes / ms / 1e6, 1), "frac": round(nbytes / ms / 1e6 / peak, 4), "peak_GBps": peak,
           "peak_source": peak_kind, "create_s": round(t_create, 2), "launch": info,
           "max_err_in_bound_units": round(worst, 4)}
    del R, d_in, d_out
    torch.cuda.empty_cache()
    return res


CONTROL_WIDTHS = [65536, 262144]
SCREEN_NAMES = {0: "candidate", 1: "no_reuse", 2: "ordered", 3: "remote_state"}


def run_controls_bench(C, torch, dev, synth):
    """Negative controls of the structural screen (Sec. III-D, IV-C): the row scan and the 5-point row stencil
    over 4096 x {64K, 256K} FP32, planned (the screen's verdict, the global-memory path) and timed (median of
    5, 8 B per element); the selection case by its verdict alone.  The scan's carries are ordered, K = 2(P - 1):
    its control cost is estimated from the measured work-free control kernel of the cluster launch shape at
    one exchange stage plus (P - 2) further stages, each priced at the measured difference between the two- and
    one-stage control kernels; the one-pass scan rereads nothing (T_save = 0), so dT = -T_ctrl < 0 at every P."""
    out = {"rows": ROWS, "dtype": "f32", "bytes_per_elem": 8, "shapes": [], "screen": {}}
    peak, peak_kind = measured_peak()
    for op, name in ((C.SCAN, "scan"), (C.STENCIL, "stencil"), (C.SELECT, "select"), (C.LOGSUMEXP, "logsumexp")):
        out["screen"][name] = SCREEN_NAMES[C.screen(C.dataflow(op), 16)[0]]
    w = torch.tensor([0.1, -0.2, 0.4, -0.2, 0.1], device=dev)
    for cols in CONTROL_WIDTHS:
        x = synth.outliers(ROWS, cols, seed=synth.SEED_DATA, device=dev)
        y = torch.empty_like(x)
        for op, name, kw in ((C.SCAN, "scan", {}), (C.STENCIL, "stencil", dict(weights=w))):
            plan, verdict = C.plan_control(op, ROWS, cols)
            ms = statistics.median(time_events(lambda: C.run_control(op, x, y, **kw), 5, warm=2))
            nbytes = ROWS * cols * 8
            out["shapes"].append({"op": name, "cols": cols, "verdict": SCREEN_NAMES[verdict],
                                  "path": "global, one CTA per row" if op == C.SCAN else "global",
                                  "ms": round(ms, 4), "GBps": round(nbytes / ms / 1e6, 1),
                                  "frac": round(nbytes / ms / 1e6 / peak, 4)})
        del x, y
        torch.cuda.empty_cache()
    # the scan's ordered-carry control cost, priced from the measured control kernel (FP8 launch shape: the
    # one- and two-stage control kernels share it)
    cols = CONTROL_WIDTHS[0]
    est = []
    for P in (2, 4, 8, 16):
        try:
            t1 = C.control_time(C.SOFTMAX, ROWS, cols, C.FP8_E4M3, P)
            t2 = C.control_time(C.LAYERNORM, ROWS, cols, C.FP8_E4M3, P)
            t0 = C.control_time(C.SOFTMAX, ROWS, cols, C.FP8_E4M3, 1)
        except C.CreditError:
            continue
        K = C.screen(C.dataflow(C.SCAN), P)[1]
        t_ctrl = (t1 - t0) + (K // 2 - 1) * max(0.0, t2 - t1)
        est.append({"P": P, "K": K, "T_ctrl_us": round(t_ctrl, 2), "stage_us": round(max(0.0, t2 - t1), 2),
                    "T_save_us": 0.0, "dT_us": round(-t_ctrl, 2)})
    out["scan_ordered_control"] = {"cols": cols, "per_P": est}
    out["peak_GBps"], out["peak_source"] = peak, peak_kind
    assert C.device_error() == C.OK
    return out


PATH_NAMES_SHORT = {0: "one_cta", 1: "two_pass", 2: "cluster"}


def profitability(pick_rows):
    """Paper-style profitability pairs (Sec. IV): per shape, does the analytic
    model's sign of dT (cluster picked or not) agree with the measured sign
    (best shared-memory cluster plan faster than the best non-DSMEM plan)?
    Plus N*, the smallest width where the cluster path wins, per op, predicted
    and measured."""
    agree = sum(r["analytic_cluster"] == r["measured_cluster"] for r in pick_rows)
    n_star = {}
    for r in sorted(pick_rows, key=lambda r: r["cols"]):
        d = n_star.setdefault(r["op"], {"analytic": None, "measured": None})
        if r["analytic_cluster"] and d["analytic"] is None:
            d["analytic"] = r["cols"]
        if r["measured_cluster"] and d["measured"] is None:
            d["measured"] = r["cols"]
    return {"pairs": len(pick_rows), "sign_agreement": agree, "n_star": n_star}


def run_e2e(C, torch, dev, jobs, shapes, stream, args, world=1):
    """The same step through the public host-buffer call (credit_run_host):
    every op copies its input in from pinned host memory, runs, and copies its
    output back, the library overlapping the copies of consecutive row blocks
    with the op.  Wall-clock time of whole steps (the call is synchronous),
    bracketed by barriers and taken as the max over ranks; the value counts
    every rank's rows."""
    import torch.distributed as dist
    host_x, host_g, host_b = {}, {}, {}
    for sh in shapes:
        for src, dst in ((sh["x"], host_x), (sh["g"], host_g), (sh["b"], host_b)):
            h = torch.empty(src.shape, dtype=src.dtype, pin_memory=True)
            h.copy_(src)
            dst[sh["cols"]] = h
    big = max(sh["x"].numel() for sh in shapes)
    host_y = torch.empty(big, dtype=torch.float32, pin_memory=True)
    h2d = d2h = 0
    for j in jobs:
        h2d += host_x[j["cols"]].numel() * 4 + j["cols"] * 4 * (2 if j["op"] == C.LAYERNORM else 1)
        d2h += j["y"].numel() * 4

    def step():
        for j in jobs:
            c = j["cols"]
            C.run_host(j["op"], host_x[c], host_y[: j["y"].numel()].view(j["y"].shape), gamma=host_g[c],
                       beta=host_b[c] if j["op"] == C.LAYERNORM else None)

    steps = max(1, min(args.steps, args.e2e_steps))
    step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / steps, world, device=dev)
    step_bytes = sum(j["bytes"] for j in jobs)
    value = job_value(step_bytes, world, ms)
    # the host link's own rates on this machine, for scale: 1 GiB plain copies between the same pinned
    # buffers and device tensors (the input is copied onto its own device copy, so nothing changes)
    big_cols = max(host_x, key=lambda c: host_x[c].numel())
    dj = next(j for j in jobs if j["cols"] == big_cols)
    n = min(1 << 28, host_x[big_cols].numel())
    hx, dx = host_x[big_cols].view(-1)[:n], dj["x"].view(-1)[:n]
    hy, dy = host_y[:n], dj["y"].view(-1)[:n]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def copy_rate(h2d_on, d2h_on, reps=3):
        def go():
            if h2d_on:
                with torch.cuda.stream(s_in):
                    dx.copy_(hx, non_blocking=True)
            if d2h_on:
                with torch.cuda.stream(s_out):
                    hy.copy_(dy, non_blocking=True)
        go()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            go()
        torch.cuda.synchronize()
        return round((h2d_on + d2h_on) * n * 4 * reps / (time.perf_counter() - t) / 1e9, 1)

    link = {"h2d": copy_rate(True, False), "d2h": copy_rate(False, True), "both": copy_rate(True, True)}
    return {"value": round(value, 1), "unit": "GB/s", "h2d_bytes_per_step": h2d * world,
            "d2h_bytes_per_step": d2h * world, "ms_per_step": round(ms, 3), "steps": steps,
            "api": "credit_run_host (pinned host buffers, library-planned row blocks)",
            "link_gbs": link, "frac_of_link_both": round(value / world / link["both"], 3)}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--widths", default="")
    ap.add_argument("--no-picks", action="store_true")
    ap.add_argument("--no-model", action="store_true", help="plan with the built-in heuristic")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-bwd", action="store_true", help="skip the backward-op table")
    ap.add_argument("--no-quant", action="store_true", help="skip the int8 quantisation table")
    ap.add_argument("--no-prec", action="store_true", help="skip the BF16 / FP8 softmax / log-sum-exp table")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-batch graph launch")
    ap.add_argument("--no-controls", action="store_true", help="skip the negative controls (scan, stencil)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="--impl reference: CPU seconds of the whole run, split over warm-up and timed steps")
    ap.add_argument("--case", default="", help="op:rows:cols:path:P[:retain[:fill_share[:f32|bf16|e4m3]]] -- one plan, 3 calls (for ncu)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.case:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
