"""Profiling sweep, learned-model training and pick-accuracy evaluation.

Times every legal candidate plan (one-CTA and cluster P in {2, 4, 8, 16}, each
with the slice retained in shared memory and, where that applies, in tensor
memory; cluster plans that leave SMs idle also with fill shares 0.15-0.4;
two-pass G in {1, 2, 4, 8} and the split factor) of a seeded set of shapes (rows
2^U(6,16), cols 2^U(10,20), dtype and op uniform, I/O <= a byte cap;
median of `reps` CUDA-event timings), splits the shapes 80/20, trains the
latency MLP on the GPU with the library's kernels, and reports, on the
held-out shapes, how often each planner's pick is within 5% of the measured
best candidate: the learned model, the analytic model (Eq. 7-9), and the
ablation model of Table IV.

    python -m paper_2609_01864_gb300.sweep --shapes 2000 --out DIR

writes DIR/gb300_mlp.txt (weights), DIR/sweep_gb300.csv (timings) and
DIR/sweep_gb300_summary.json.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

import numpy as np
import torch

from . import credit as C
from . import synth

DT_TORCH = {0: torch.float32, 1: torch.bfloat16, 2: torch.float8_e4m3fn}
# fill candidates of cluster plans that leave at least FILL_MIN_IDLE SMs idle
# (the library's learned planner offers the same shares)
FILL_SHARES = (0.15, 0.2, 0.3, 0.4)
FILL_MIN_IDLE = 16
FILL_MIN_ROWS = 64


def candidates(op, rows, cols, dtype, x, y, sc, osc, gamma, beta):
    out = []
    kw = dict(rows=rows, cols=cols, in_dtype=dtype, out_dtype=C.F32 if op == C.LOGSUMEXP else dtype,
              in_scale=sc, out_scale=osc, gamma=gamma, beta=beta)
    sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    for P in (1, 2, 4, 8, 16):
        legal = []
        for retain in (C.RETAIN_SMEM, C.RETAIN_TMEM):
            p = C.make_plan(C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER, P, retain=retain)
            if C.plan_check(op, x, y, p, **kw) == C.OK:
                out.append((C.PATH_ONE_CTA if P == 1 else C.PATH_CLUSTER, P, P, retain, 0.0, p))
                legal.append((retain, p))
        # fills of a cluster plan that leaves SMs idle (the tensor-memory tier when it applies)
        if P > 1 and legal and rows >= FILL_MIN_ROWS:
            retain, p = legal[-1]
            if sm - P * C.max_clusters(op, x, y, p, **kw) >= FILL_MIN_IDLE:
                for f in FILL_SHARES:
                    out.append((C.PATH_CLUSTER, P, P, retain, f, C.make_plan(C.PATH_CLUSTER, P, retain=retain,
                                                                              fill_share=f)))
    isz = {0: 4, 1: 2, 2: 1}[dtype]
    groups = cols * isz // 16
    Gs = [G for G in (1, 2, 4, 8) if G == 1 or groups // G >= 1024]
    g_auto = two_pass_split(rows, cols, dtype)
    if g_auto > 1 and g_auto not in Gs:
        Gs.append(g_auto)
    for G in Gs:
        out.append((C.PATH_TWO_PASS, 1, G, C.RETAIN_AUTO, 0.0, C.make_plan(C.PATH_TWO_PASS, ctas_per_row=G)))
    return out, kw


def two_pass_split(rows, cols, dtype, sm_count=None):
    """Mirror of the library's split rule (enough CTAs for 4 waves, >= 1024
    16-byte groups per CTA)."""
    if sm_count is None:
        sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    isz = {0: 4, 1: 2, 2: 1}[dtype]
    target = 4 * sm_count
    if rows >= target:
        return 1
    G = -(-target // rows)
    gmax = max(1, (cols * isz // 16) // 1024)
    return int(max(1, min(G, gmax, 1024)))


def time_plan(fn, reps):
    for _ in range(2):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record()
        fn()
        b.record()
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) * 1e3 for a, b in ev)


def run_sweep(shapes, reps, cap_bytes, log=None):
    dev = torch.device("cuda", torch.cuda.current_device())
    buf_in = torch.empty(cap_bytes, dtype=torch.uint8, device=dev)
    buf_out = torch.empty(cap_bytes, dtype=torch.uint8, device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(synth.SEED_SWEEP)
    # inputs: N(0, 1) floats written through each dtype's view of the same buffer
    max_cols = max(s[3] for s in shapes)
    max_rows = max(s[2] for s in shapes)
    gamma, beta = synth.gamma_beta(max_cols, device=dev)
    scales = torch.ones(max_rows, device=dev)
    oscales = torch.empty(max_rows, device=dev)
    rows_out = []
    t0 = time.time()
    for si, (op, dt, rows, cols) in enumerate(shapes):
        isz = {0: 4, 1: 2, 2: 1}[dt]
        x = buf_in[: rows * cols * isz].view(DT_TORCH[dt]).view(rows, cols)
        src = torch.randn(rows, cols, device=dev, generator=g) if rows * cols * 4 <= 2 ** 31 else None
        if src is not None:
            x.copy_(src.clamp_(-8, 8).to(DT_TORCH[dt]))
            del src
        else:
            x.view(torch.uint8).fill_(0x3c)
        y = buf_out[: rows * cols * 4].view(torch.float32)
        cands, kw = candidates(op, rows, cols, dt, x, y, scales[:rows], oscales[:rows],
                               gamma[:cols] if op in (2, 3) else None, beta[:cols] if op == 2 else None)
        times = []
        for path, P, G, retain, fill, plan in cands:
            us = time_plan(lambda: C.run_ex(op, x, y, plan=plan, **kw), reps)
            times.append((path, P, G, retain, fill, us))
        for path, P, G, retain, fill, us in times:
            rows_out.append(dict(shape=si, op=op, dtype=dt, rows=rows, cols=cols, path=path, P=P, G=G,
                                 retain=retain, fill=fill, us=us))
        if log and si % 100 == 0:
            print(f"shape {si}/{len(shapes)} {time.time() - t0:.0f}s", file=log, flush=True)
    assert C.device_error() == C.OK
    return rows_out


CSV_HEADER = "shape,op,dtype,rows,cols,path,P,G,retain,fill,us"


def write_csv(path, rows):
    """One line per timed candidate (times in microseconds)."""
    with open(path, "w") as f:
        f.write(CSV_HEADER + "\n")
        for r in rows:
            f.write(f"{r['shape']},{r['op']},{r['dtype']},{r['rows']},{r['cols']},{r['path']},{r['P']},{r['G']},"
                    f"{r['retain']},{r['fill']:g},{r['us']:.3f}\n")


def read_csv(path):
    """Timings written by write_csv, and the two older forms: 9 columns (no
    retention column: cluster and one-CTA plans staged in shared memory) and
    10 columns (no fill column: no fill)."""
    rows = []
    with open(path) as f:
        next(f)
        for line in f:
            v = line.strip().split(",")
            if len(v) == 9:
                v = v[:8] + [str(C.RETAIN_SMEM if int(v[5]) != C.PATH_TWO_PASS else C.RETAIN_AUTO)] + v[8:]
            if len(v) == 10:
                v = v[:9] + ["0"] + v[9:]
            if len(v) != 11:
                raise ValueError(f"{path}: bad timing line {line.strip()!r}")
            sh, op, dt, r, c, path_, P, G, retain, fill, us = v
            rows.append(dict(shape=int(sh), op=int(op), dtype=int(dt), rows=int(r), cols=int(c), path=int(path_),
                             P=int(P), G=int(G), retain=int(retain), fill=float(fill), us=float(us)))
    return rows


def features_of(r):
    out_dt = C.F32 if r["op"] == C.LOGSUMEXP else r["dtype"]
    return C.mlp_features(r["op"], r["dtype"], out_dt, r["rows"], r["cols"], r["path"], r["P"], r["G"],
                          r.get("retain", 0), r.get("fill", 0.0))


FILL_TIE_LOG2 = 0.01  # the learned planner's tie-break (kFillTieLog2 in csrc/credit_mlp.cu)


def learned_pick(cand):
    """The learned planner's choice among a shape's measured candidates: the lowest prediction or, within
    FILL_TIE_LOG2 of it, the lowest one without a fill."""
    lo = min(c["pred_log2us"] for c in cand)
    nofill = [c for c in cand if c.get("fill", 0.0) == 0.0 and c["pred_log2us"] <= lo + FILL_TIE_LOG2]
    return min(nofill or cand, key=lambda c: c["pred_log2us"])


def evaluate(rows, test_shapes):
    by_shape = {}
    for r in rows:
        by_shape.setdefault(r["shape"], []).append(r)
    res = {"learned": 0, "analytic": 0, "ablation": 0, "always_two_pass": 0, "always_best_non_dsmem": 0}
    n = 0
    feats, owners = [], []
    for s in test_shapes:
        for r in by_shape.get(s, []):
            feats.append(features_of(r))
            owners.append(r)
    pred = C.mlp_predict(np.stack(feats)) if feats else []
    for r, pr in zip(owners, pred):
        r["pred_log2us"] = float(pr)
    for s in test_shapes:
        cand = by_shape.get(s)
        if not cand:
            continue
        n += 1
        best = min(c["us"] for c in cand)
        ok = lambda c: c["us"] <= 1.05 * best  # noqa: E731
        learned = learned_pick(cand)
        res["learned"] += ok(learned)
        r0 = cand[0]
        for name, env in (("analytic", "analytic"), ("ablation", "ablation")):
            os.environ["CREDIT_MODEL"] = env
            p = C.plan(r0["op"], r0["rows"], r0["cols"], r0["dtype"])
            os.environ.pop("CREDIT_MODEL", None)
            match = [c for c in cand if c["path"] == p.path and (c["P"] == p.cluster_size if p.path != C.PATH_TWO_PASS
                                                                  else c["G"] == p.ctas_per_row)
                     and (p.path == C.PATH_TWO_PASS or c.get("retain", 0) == p.retain)
                     and abs(c.get("fill", 0.0) - p.fill_share) < 1e-6]
            res[name] += ok(match[0]) if match else 0
        tp = [c for c in cand if c["path"] == C.PATH_TWO_PASS and c["G"] == 1]
        res["always_two_pass"] += ok(tp[0]) if tp else 0
        nd = [c for c in cand if c["path"] != C.PATH_CLUSTER]
        res["always_best_non_dsmem"] += ok(min(nd, key=lambda c: c["us"])) if nd else 0
    return {k: v / max(1, n) for k, v in res.items()}, n


def reusable_timings(old_rows, shapes):
    """Timings of an earlier sweep that still describe shape i of `shapes` (every row recorded for id i has the
    same op, dtype, rows and cols), and the ids that must be timed again (sorted)."""
    old = {}
    for r in old_rows:
        old.setdefault(r["shape"], []).append(r)
    keep = [i for i, (op, dt, nr, nc) in enumerate(shapes)
            if i in old and all((r["op"], r["dtype"], r["rows"], r["cols"]) == (op, dt, nr, nc) for r in old[i])]
    kept_ids = set(keep)
    return [r for i in keep for r in old[i]], [i for i in range(len(shapes)) if i not in kept_ids]


def eval_only(args) -> int:
    """Pick accuracies of the loaded learned model and of the analytic / ablation planners on the held-out
    split of the committed sweep, written back into the summary (the planners can change after a sweep)."""
    from . import build as B
    B.build()
    C.init()
    C.load_model(args.calib)
    path = os.path.join(args.out, "sweep_gb300_summary.json")
    with open(path) as f:
        summary = json.load(f)
    rows = read_csv(os.path.join(args.out, "sweep_gb300.csv"))
    _, test = synth.split_by_shape(summary["shapes"])
    acc, n = evaluate(rows, test)
    if n != summary["test_shapes"]:
        raise SystemExit(f"held-out shapes {n} != {summary['test_shapes']} in the summary")
    summary["pick_accuracy"] = acc
    with open(path, "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps({"pick_accuracy": acc, "test_shapes": n}))
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", type=int, default=2000)
    ap.add_argument("--reps", type=int, default=15)
    ap.add_argument("--cap-gib", type=float, default=16.0)
    ap.add_argument("--epoch-grid", type=int, nargs="+", default=[50, 100, 200, 400, 800])
    ap.add_argument("--members", type=int, default=5, help="ensemble size of the learned model")
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data"))
    ap.add_argument("--calib", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "data",
                                                    "gb300.calib"))
    ap.add_argument("--from-csv", default="", help="retrain and evaluate from an earlier sweep's timings")
    ap.add_argument("--extra-shapes", type=int, default=300,
                    help="training-only shapes from the wide-row corner (rows 2^U(10,14), cols 2^U(14,20)); cols "
                         "as drawn, rounded to a power of two, rounded down to a multiple of 16, in turn")
    ap.add_argument("--reuse-csv", default="",
                    help="take the timings of shapes identical to an earlier sweep's (same id, op, dtype, rows, "
                         "cols) from its CSV and time only the others (the kernels must be the same)")
    ap.add_argument("--target", default="relative", choices=["relative", "absolute"],
                    help="log2 latency relative to the shape's mean over its candidates, or absolute")
    ap.add_argument("--eval-only", action="store_true",
                    help="no sweep, no training: evaluate the committed model and the planner rules on the held-out "
                         "shapes of the committed timings and update the summary's pick accuracies")
    args = ap.parse_args(argv)
    if args.eval_only:
        return eval_only(args)
    from . import build as B
    B.build()
    C.init()
    try:
        C.load_model(args.calib)
    except C.CreditError as e:  # the calibration loads before the weights it names; stale weights are replaced below
        print(f"note: {e}", file=sys.stderr)
    cap = int(args.cap_gib * 2 ** 30)
    shapes = synth.sweep_shapes(args.shapes, cap_bytes=cap)
    # training-only shapes from the wide-row corner (thousands of rows of 16K-1M columns, up to the byte cap),
    # which the log-uniform draw above reaches rarely: shape ids from len(shapes) on, never in the held-out split
    extra = synth.sweep_shapes(args.extra_shapes, seed=synth.SEED_SWEEP + 11, cap_bytes=cap,
                               rows_log2=(10.0, 14.0), cols_log2=(14.0, 20.0),
                               col_modes=("any", "pow2", "align16")) if args.extra_shapes > 0 else []
    t0 = time.time()
    if args.from_csv:
        rows = read_csv(args.from_csv)
        rows = [r for r in rows if r["shape"] < len(shapes) + len(extra)]
    elif args.reuse_csv:
        allshapes = shapes + extra
        kept, todo = reusable_timings(read_csv(args.reuse_csv), allshapes)
        print(f"reusing {len(allshapes) - len(todo)} shapes, timing {len(todo)}", file=sys.stderr)
        new_rows = run_sweep([allshapes[i] for i in todo], args.reps, cap, log=sys.stderr)
        for r in new_rows:
            r["shape"] = todo[r["shape"]]
        rows = kept + new_rows
    else:
        rows = run_sweep(shapes + extra, args.reps, cap, log=sys.stderr)
    t_sweep = time.time() - t0
    train, test = synth.split_by_shape(len(shapes))
    extra_ids = list(range(len(shapes), len(shapes) + len(extra)))

    # targets: log2 latency, by default relative to the mean over the shape's candidates -- the planner ranks
    # the candidates of one shape, so the level of a shape carries no information for it, and removing it
    # leaves the network the within-shape differences to learn (the planner anchors absolute predictions on
    # the calibration's baseline timing T_B)
    level = {}
    for r in rows:
        level.setdefault(r["shape"], []).append(np.log2(r["us"]))
    level = {k: float(np.mean(v)) for k, v in level.items()}

    def xy(shape_set):
        X = np.stack([features_of(r) for r in rows if r["shape"] in shape_set])
        y = np.array([np.log2(r["us"]) - (level[r["shape"]] if args.target == "relative" else 0.0)
                      for r in rows if r["shape"] in shape_set], dtype=np.float32)
        return X, y

    t1 = time.time()
    # epochs chosen on a validation split of the training shapes (the held-out
    # test shapes are used once, for the final report)
    fit_idx, val_idx = synth.split_by_shape(len(train), seed=synth.SEED_SWEEP + 7, train_frac=0.85)
    fit_set, val_set = {train[i] for i in fit_idx} | set(extra_ids), [train[i] for i in val_idx]
    Xf, yf = xy(fit_set)
    val_acc = {}
    for ep in args.epoch_grid:
        C.mlp_train_ensemble(Xf, yf, members=args.members, epochs=ep, batch=256, lr=2e-3, seed=0)
        val_acc[ep] = evaluate(rows, val_set)[0]["learned"]
    epochs = max(args.epoch_grid, key=lambda e: (val_acc[e], -e))
    Xtr, ytr = xy(set(train) | set(extra_ids))
    curve = C.mlp_train_ensemble(Xtr, ytr, members=args.members, epochs=epochs, batch=256, lr=2e-3, seed=0)
    t_train = time.time() - t1
    acc, n_test = evaluate(rows, test)
    os.makedirs(args.out, exist_ok=True)
    C.mlp_save(os.path.join(args.out, "gb300_mlp.txt"))
    csv_out = os.path.join(args.out, "sweep_gb300.csv")
    if args.from_csv and os.path.abspath(args.from_csv) == os.path.abspath(csv_out):
        csv_out += ".new"
    write_csv(csv_out, rows)
    summary = {"shapes": len(shapes), "timings": len(rows), "train_shapes": len(train), "test_shapes": n_test,
               "extra_train_shapes": len(extra),
               "extra_distribution": "rows 2^U(10,14), cols 2^U(14,20) as drawn / nearest power of two / down to a "
                                     "multiple of 16 in turn, dtype and op uniform, I/O <= the cap",
               "pick_rule": "pick within 5% of the measured best candidate", "pick_accuracy": acc,
               "train_loss_first_last": [float(curve[0]), float(curve[-1])], "sweep_s": round(t_sweep, 1),
               "epochs": epochs, "validation_accuracy_by_epochs": val_acc,
               "train_s": round(t_train, 1), "reps": args.reps, "cap_gib": args.cap_gib,
               "members": args.members, "target": args.target}
    with open(os.path.join(args.out, "sweep_gb300_summary.json"), "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
