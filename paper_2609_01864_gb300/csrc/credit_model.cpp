// credit_model.cpp -- profitability model of CREDIT Sec. III-D and its
// calibration.
//
// The analytic model scores the cluster path against the selected non-DSMEM
// baseline with one measured baseline time T_B(M, N) (Eq. 7), the control
// kernel's excess time T_ctrl(M, N, P), and the measured shared-memory and
// DSMEM rates (Eq. 8): dT = T_save - T_ctrl - T_replay - T_deposit - T_DSM
// (Eq. 9).  The cluster path is picked for the P with the largest dT when
// that is positive; otherwise the baseline: the one-CTA staged kernel when
// the row fits one CTA (Eq. 3), else the two-pass reread kernel (Sec. IV-A).
// Scalar-output reductions have b_reread = 0 and are rejected by
// construction (Sec. III-D, last paragraph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "credit_model.h"

namespace credit {

namespace {

constexpr int kMaxDev = 64;
const int kPs[4] = {2, 4, 8, 16};

struct TbCell {
    long long rows, cols;
    double us;
    double bytes_per_us;  // rows * cols * b_B / us
};
struct CtrlCell {
    long long rows, cols;
    int P;
    double us_p, us_1;
};
struct Calib {
    bool loaded = false;
    credit_microbench_t mb{};
    double hbm_gbs = 0.0;
    std::map<int, std::vector<TbCell>> tb;     // key op * 8 + dtype
    std::map<int, std::vector<CtrlCell>> ctrl;  // key dtype
    std::string mlp_path;   // as written in the file: absolute, or relative to the file's directory
    std::string mlp_dir;    // the directory of the file it was read from (load time only)
};
Calib g_cal[kMaxDev];
std::mutex g_cal_mu;

int tb_key(int op, int dt) { return op * 8 + dt; }

// Static analysis of the selected baseline (bytes per element).
struct Bytes {
    double b_B, b_reread, b_keep, b_in, q_sum;
    bool one_cta;  // baseline is the one-CTA staged kernel
};

}  // namespace

// ------------------------------------------------------------------ Eq. 7-9
static void eval_terms(const credit_model_inputs &in, credit_model_terms &o) {
    std::memset(&o, 0, sizeof(o));
    const double M = in.M, N = in.N, P = in.P;
    o.W = std::ceil(M / std::max(1.0, in.active_clusters));
    o.B_eff_gbs = in.T_B_us > 0 ? M * N * in.b_B / in.T_B_us * 1e-3 : 0.0;  // bytes/us -> GB/s
    const double slice = std::ceil(N / P) * in.b_keep;
    const double fB_r = in.f_mhz * in.B_smem_read, fB_w = in.f_mhz * in.B_smem_store;
    const double fB_d = in.f_mhz * in.B_dsm_store;
    o.T_replay_us = fB_r > 0 ? o.W * slice / fB_r : 0.0;
    o.T_dsm_us = fB_d > 0 ? in.s_bytes * o.W * (P - 1.0) * in.q_sum / fB_d : 0.0;
    o.T_smem_w_us = fB_w > 0 ? o.W * slice / fB_w : 0.0;
    if (in.ablation) {
        o.T_save_us = in.B_peak_gbs > 0 ? M * N * in.b_reread / (in.B_peak_gbs * 1e3) : 0.0;
        o.T_input_us = 0.0;
        o.T_deposit_us = o.T_smem_w_us;
    } else {
        o.T_save_us = in.b_B > 0 ? in.T_B_us * in.b_reread / in.b_B : 0.0;
        o.T_input_us = o.B_eff_gbs > 0 ? M * N * in.b_in / (o.B_eff_gbs * 1e3) : 0.0;
        o.T_deposit_us = std::max(0.0, o.T_smem_w_us - o.T_input_us);
    }
    o.dT_us = o.T_save_us - in.T_ctrl_us - o.T_replay_us - o.T_deposit_us - o.T_dsm_us;
}

static Bytes static_bytes(int op, int tin, int tout, bool one_cta) {
    const double bi = dtype_size(tin), bo = op == 1 ? 0.0 : dtype_size(tout);
    Bytes b{};
    b.b_in = bi;
    b.b_keep = bi;
    b.one_cta = one_cta;
    if (op == 1) {  // log-sum-exp: one streaming pass, nothing to reuse
        b.b_B = bi;
        b.b_reread = 0.0;
    } else if (one_cta) {
        b.b_B = bi + bo;
        b.b_reread = 0.0;
    } else {
        b.b_B = 2.0 * bi + bo;
        b.b_reread = bi;
    }
    b.q_sum = (op == 3) ? 1.0 : 2.0;
    if ((op == 2 || op == 3) && tout == 2) b.q_sum += 1.0;  // FP8-output amax stage
    return b;
}

// Interpolated baseline bandwidth (bytes/us), bilinear in log2 of rows and
// cols over the calibration grid, clamped at its edges.
static double tb_bytes_per_us(const Calib &cal, int op, int dt, long long M, long long N) {
    auto it = cal.tb.find(tb_key(op, dt));
    if (it == cal.tb.end() || it->second.empty()) return 0.0;
    const auto &cells = it->second;
    std::vector<long long> R, Cc;
    for (const auto &c : cells) {
        R.push_back(c.rows);
        Cc.push_back(c.cols);
    }
    std::sort(R.begin(), R.end());
    R.erase(std::unique(R.begin(), R.end()), R.end());
    std::sort(Cc.begin(), Cc.end());
    Cc.erase(std::unique(Cc.begin(), Cc.end()), Cc.end());
    auto bracket = [](const std::vector<long long> &v, double x, int &i0, int &i1, double &t) {
        if (x <= v.front()) {
            i0 = i1 = 0;
            t = 0;
            return;
        }
        if (x >= v.back()) {
            i0 = i1 = static_cast<int>(v.size()) - 1;
            t = 0;
            return;
        }
        i1 = 1;
        while (v[i1] < x) ++i1;
        i0 = i1 - 1;
        t = (std::log2(x) - std::log2(static_cast<double>(v[i0]))) /
            (std::log2(static_cast<double>(v[i1])) - std::log2(static_cast<double>(v[i0])));
    };
    int r0, r1, c0, c1;
    double tr, tc;
    bracket(R, static_cast<double>(M), r0, r1, tr);
    bracket(Cc, static_cast<double>(N), c0, c1, tc);
    // value at a grid point; a missing cell (skipped for its size) takes the
    // nearest measured cell of the same column width, else of any width
    auto at = [&](int ri, int ci) -> double {
        const TbCell *best = nullptr;
        long long bestd = -1;
        for (const auto &c : cells) {
            if (c.cols != Cc[ci]) continue;
            const long long d = std::llabs(c.rows - R[ri]);
            if (!best || d < bestd) {
                best = &c;
                bestd = d;
            }
        }
        if (!best)
            for (const auto &c : cells) {
                const long long d = std::llabs(c.cols - Cc[ci]) + std::llabs(c.rows - R[ri]);
                if (!best || d < bestd) {
                    best = &c;
                    bestd = d;
                }
            }
        return std::log2(best->bytes_per_us);
    };
    const double v = (1 - tr) * ((1 - tc) * at(r0, c0) + tc * at(r0, c1)) + tr * ((1 - tc) * at(r1, c0) + tc * at(r1, c1));
    return std::exp2(v);
}

// T_ctrl excess (us) for (dtype, M, N, P): nearest calibrated cols, log-linear in rows.
static double ctrl_excess_us(const Calib &cal, int dt, long long M, long long N, int P) {
    auto it = cal.ctrl.find(dt);
    if (it == cal.ctrl.end()) return 0.0;
    const CtrlCell *lo = nullptr, *hi = nullptr;
    long long best_cols = -1;
    double best_d = 1e30;
    for (const auto &c : it->second) {
        if (c.P != P) continue;
        const double d = std::fabs(std::log2(static_cast<double>(c.cols)) - std::log2(static_cast<double>(N)));
        if (d < best_d) {
            best_d = d;
            best_cols = c.cols;
        }
    }
    if (best_cols < 0) return 0.0;
    for (const auto &c : it->second) {
        if (c.P != P || c.cols != best_cols) continue;
        if (c.rows <= M && (!lo || c.rows > lo->rows)) lo = &c;
        if (c.rows >= M && (!hi || c.rows < hi->rows)) hi = &c;
    }
    auto ex = [](const CtrlCell *c) { return std::max(0.0, c->us_p - c->us_1); };
    if (!lo) return ex(hi);
    if (!hi) return ex(lo) * static_cast<double>(M) / static_cast<double>(lo->rows);  // grows ~ with waves
    if (lo == hi) return ex(lo);
    const double t = (std::log2(static_cast<double>(M)) - std::log2(static_cast<double>(lo->rows))) /
                     (std::log2(static_cast<double>(hi->rows)) - std::log2(static_cast<double>(lo->rows)));
    return (1 - t) * ex(lo) + t * ex(hi);
}

int two_pass_split(int sm_count, long long rows, long long cols, int isz);

// Selected non-DSMEM baseline (Sec. IV-A): the one-CTA staged kernel when
// the row fits one CTA, else the two-pass reread kernel.
static void baseline_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                          credit_plan_t *p) {
    std::memset(p, 0, sizeof(*p));
    RingCfg rc;
    if (op != 1 && ring_config(di, cols, dtype_size(tin), 1, 0, 0, 0, 0, 0, &rc) &&
        ring_max_clusters(device, op, tin, tout, 1, rc.threads, rc.smem) > 0) {
        p->path = CREDIT_PATH_ONE_CTA;
        p->cluster_size = 1;
        p->ctas_per_row = 1;
        p->smem_bytes = rc.smem;
        p->retain = CREDIT_RETAIN_SMEM;  // the paper's staging
    } else {
        p->path = CREDIT_PATH_TWO_PASS;
        p->cluster_size = 1;
        p->ctas_per_row = two_pass_split(di.sm_count, rows, cols, dtype_size(tin));
    }
}

bool baseline_estimate(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                       credit_plan_t *base, double *T_B_us) {
    baseline_plan(di, device, op, rows, cols, tin, tout, base);
    *T_B_us = 0.0;
    if (device < 0 || device >= kMaxDev) return false;
    Calib cal;
    {
        std::lock_guard<std::mutex> lk(g_cal_mu);
        if (!g_cal[device].loaded) return false;
        cal = g_cal[device];
    }
    const Bytes b = static_bytes(op, tin, tout, base->path == CREDIT_PATH_ONE_CTA);
    const double bw = tb_bytes_per_us(cal, op, tin, rows, cols);
    if (!(bw > 0)) return false;
    *T_B_us = static_cast<double>(rows) * cols * b.b_B / bw;
    return true;
}

// Score every legal P with Eq. 7-9.  Returns false without calibration.
bool analytic_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                   int ablation, credit_plan_t *p, double *best_dT) {
    if (device < 0 || device >= kMaxDev) return false;
    Calib cal;
    {
        std::lock_guard<std::mutex> lk(g_cal_mu);
        if (!g_cal[device].loaded) return false;
        cal = g_cal[device];
    }
    credit_plan_t base;
    baseline_plan(di, device, op, rows, cols, tin, tout, &base);
    const Bytes b = static_bytes(op, tin, tout, base.path == CREDIT_PATH_ONE_CTA);
    const double bw = tb_bytes_per_us(cal, op, tin, rows, cols);  // baseline bytes/us
    const double T_B = bw > 0 ? static_cast<double>(rows) * cols * b.b_B / bw : 0.0;
    *p = base;
    p->source = 0;
    p->predicted_us = static_cast<float>(T_B);
    double best = 0.0;
    int bestP = 0;
    RingCfg best_rc{};
    // the retention tier of each P follows the library's AUTO rule: tensor memory for slices above
    // kTmAutoMinSlice where the op has a reuse pass that tier supports (its own Eq. 3 capacity and
    // occupancy), else the shared-memory ring the paper's model describes
    const int isz = dtype_size(tin);
    const bool tm_op = op != 1 && !(tout == 2 && (op == 2 || op == 3));
    bool best_tm = false;
    for (int k = 0; k < 4 && T_B > 0; ++k) {
        const int P = kPs[k];
        RingCfg rc;
        int A = 0;
        bool tm = false;
        const long long slice = (cols * isz / 16 + P - 1) / P * 16;
        if (tm_op && slice > kTmAutoMinSlice && ring_config_tm(di, cols, isz, P, 0, 0, 0, &rc) &&
            (A = ring_max_clusters(device, op, tin, tout, P, rc.threads, rc.smem, true)) > 0) {
            tm = true;
        } else {
            if (!ring_config(di, cols, isz, P, 0, 0, 0, 0, 0, &rc)) continue;  // Eq. 3
            A = ring_max_clusters(device, op, tin, tout, P, rc.threads, rc.smem);
        }
        if (A <= 0) continue;
        credit_model_inputs in{};
        in.M = static_cast<double>(rows);
        in.N = static_cast<double>(cols);
        in.P = P;
        in.T_B_us = T_B;
        double tc = ctrl_excess_us(cal, tin, rows, cols, P);
        if (b.q_sum > 2.0 || (op == 3 && b.q_sum > 1.0)) tc *= 2.0;  // second exchange stage
        in.T_ctrl_us = tc;
        in.b_B = b.b_B;
        in.b_reread = b.b_reread;
        in.b_keep = b.b_keep;
        in.b_in = b.b_in;
        in.s_bytes = 4.0;
        in.q_sum = b.q_sum;
        in.active_clusters = A;
        in.f_mhz = cal.mb.sm_clock_mhz;
        in.B_smem_read = cal.mb.rate_local_read;
        in.B_smem_store = cal.mb.rate_local_store;
        in.B_dsm_store = cal.mb.rate_remote_store[k];
        in.B_peak_gbs = cal.hbm_gbs;
        in.ablation = ablation;
        credit_model_terms t;
        eval_terms(in, t);
        if (t.dT_us > best) {
            best = t.dT_us;
            bestP = P;
            best_rc = rc;
            best_tm = tm;
        }
    }
    if (bestP > 0) {
        p->path = CREDIT_PATH_CLUSTER;
        p->cluster_size = bestP;
        p->ctas_per_row = bestP;
        p->smem_bytes = best_rc.smem;
        p->retain = best_tm ? CREDIT_RETAIN_TMEM : CREDIT_RETAIN_SMEM;
        p->predicted_us = static_cast<float>(T_B - best);
    }
    if (best_dT) *best_dT = best;
    return true;
}

// Planner selection: CREDIT_MODEL=analytic | ablation | learned; unset means
// the learned model when its weights are loaded, else the analytic model.
// The analytic model also judges the learned pick: a cluster plan for an op
// whose structural screen rejects the cluster path (no reread to save:
// scalar-output reductions, Sec. III-D) is replaced by the learned model's
// best non-cluster candidate.
bool model_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                credit_plan_t *p) {
    const char *m = std::getenv("CREDIT_MODEL");
    const bool analytic = m && !std::strcmp(m, "analytic");
    const int ablation = (m && !std::strcmp(m, "ablation")) ? 1 : 0;
    if (!analytic && !ablation && learned_plan(di, device, op, rows, cols, tin, tout, p)) {
        if (p->path == CREDIT_PATH_CLUSTER && static_bytes(op, tin, tout, false).b_reread == 0.0)
            learned_plan_no_cluster(di, device, op, rows, cols, tin, tout, p);
        return true;
    }
    return analytic_plan(di, device, op, rows, cols, tin, tout, ablation, p, nullptr);
}

// ------------------------------------------------------------------ file I/O
// "dir/" of "dir/name" ("" for a bare name), an absolute form of a path (the
// path itself if it cannot be resolved), and whether two directories are one.
static std::string dir_of(const char *path) {
    const std::string s(path);
    const size_t k = s.find_last_of('/');
    return k == std::string::npos ? std::string() : s.substr(0, k + 1);
}
static std::string absolute(const std::string &p) {
    char buf[PATH_MAX];
    return realpath(p.c_str(), buf) ? std::string(buf) : p;
}
static bool same_dir(const std::string &a, const std::string &b) {
    return absolute(a.empty() ? "." : a) == absolute(b.empty() ? "." : b);
}

static bool write_calib(const char *path, const Calib &c, const DeviceInfo &di) {
    FILE *f = std::fopen(path, "w");
    if (!f) return false;
    std::fprintf(f, "credit-calibration 1\n");
    std::fprintf(f, "device sm_count %d smem_optin %lld cc %d.%d\n", di.sm_count, di.smem_optin, di.cc_major,
                 di.cc_minor);
    const auto &m = c.mb;
    std::fprintf(f, "clock_mhz %.3f\n", m.sm_clock_mhz);
    std::fprintf(f, "latency %.4f %.4f\n", m.lat_local_cycles, m.lat_remote_cycles);
    std::fprintf(f, "sync %.3f %.3f %.3f %.3f\n", m.sync_cycles[0], m.sync_cycles[1], m.sync_cycles[2],
                 m.sync_cycles[3]);
    std::fprintf(f, "rates %.4f %.4f %.4f\n", m.rate_local_read, m.rate_local_store, m.rate_remote_read);
    std::fprintf(f, "remote_store %.4f %.4f %.4f %.4f\n", m.rate_remote_store[0], m.rate_remote_store[1],
                 m.rate_remote_store[2], m.rate_remote_store[3]);
    std::fprintf(f, "distinct_sms %d\n", m.distinct_sms);
    std::fprintf(f, "hbm_gbs %.1f\n", c.hbm_gbs);
    for (const auto &kv : c.tb)
        for (const auto &t : kv.second)
            std::fprintf(f, "tb %d %d %lld %lld %.4f\n", kv.first / 8, kv.first % 8, t.rows, t.cols, t.us);
    for (const auto &kv : c.ctrl)
        for (const auto &t : kv.second)
            std::fprintf(f, "tctrl %d %lld %lld %d %.4f %.4f\n", kv.first, t.rows, t.cols, t.P, t.us_p, t.us_1);
    if (!c.mlp_path.empty()) std::fprintf(f, "mlp %s\n", c.mlp_path.c_str());
    return std::fclose(f) == 0;
}

static bool read_calib(const char *path, Calib &c) {
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool header = false;
    while (std::fgets(line, sizeof(line), f)) {
        char key[64] = {0};
        if (std::sscanf(line, "%63s", key) != 1) continue;
        auto &m = c.mb;
        if (!std::strcmp(key, "credit-calibration")) header = true;
        else if (!std::strcmp(key, "clock_mhz")) std::sscanf(line, "%*s %lf", &m.sm_clock_mhz);
        else if (!std::strcmp(key, "latency")) std::sscanf(line, "%*s %lf %lf", &m.lat_local_cycles, &m.lat_remote_cycles);
        else if (!std::strcmp(key, "sync"))
            std::sscanf(line, "%*s %lf %lf %lf %lf", &m.sync_cycles[0], &m.sync_cycles[1], &m.sync_cycles[2],
                        &m.sync_cycles[3]);
        else if (!std::strcmp(key, "rates"))
            std::sscanf(line, "%*s %lf %lf %lf", &m.rate_local_read, &m.rate_local_store, &m.rate_remote_read);
        else if (!std::strcmp(key, "remote_store"))
            std::sscanf(line, "%*s %lf %lf %lf %lf", &m.rate_remote_store[0], &m.rate_remote_store[1],
                        &m.rate_remote_store[2], &m.rate_remote_store[3]);
        else if (!std::strcmp(key, "distinct_sms")) std::sscanf(line, "%*s %d", &m.distinct_sms);
        else if (!std::strcmp(key, "hbm_gbs")) std::sscanf(line, "%*s %lf", &c.hbm_gbs);
        else if (!std::strcmp(key, "tb")) {
            int op, dt;
            TbCell t{};
            if (std::sscanf(line, "%*s %d %d %lld %lld %lf", &op, &dt, &t.rows, &t.cols, &t.us) == 5 && t.us > 0) {
                const int tout = op == 1 ? 0 : dt;
                const Bytes b = static_bytes(op, dt, tout, false);
                (void)b;
                c.tb[tb_key(op, dt)].push_back(t);
            }
        } else if (!std::strcmp(key, "tctrl")) {
            int dt;
            CtrlCell t{};
            if (std::sscanf(line, "%*s %d %lld %lld %d %lf %lf", &dt, &t.rows, &t.cols, &t.P, &t.us_p, &t.us_1) == 6)
                c.ctrl[dt].push_back(t);
        } else if (!std::strcmp(key, "mlp")) {
            char p[900];
            if (std::sscanf(line, "%*s %899s", p) == 1) c.mlp_path = p;
        }
    }
    std::fclose(f);
    return header && c.mb.sm_clock_mhz > 0;
}

// bytes_per_us of each baseline cell needs the baseline's b_B, which depends
// on whether the row fits one CTA on this device.
static void finish_calib(const DeviceInfo &di, Calib &c) {
    for (auto &kv : c.tb) {
        const int op = kv.first / 8, dt = kv.first % 8;
        const int tout = op == 1 ? 0 : dt;
        for (auto &t : kv.second) {
            RingCfg rc;
            const bool one = op != 1 && ring_config(di, t.cols, dtype_size(dt), 1, 0, 0, 0, 0, 0, &rc);
            const Bytes b = static_bytes(op, dt, tout, one);
            t.bytes_per_us = static_cast<double>(t.rows) * t.cols * b.b_B / t.us;
        }
    }
    c.loaded = true;
}

}  // namespace credit

using namespace credit;

extern "C" {

credit_status credit_model_eval(const credit_model_inputs *in, credit_model_terms *out) {
    if (!in || !out || in->M <= 0 || in->N <= 0 || in->P < 1) return CREDIT_ERR_INVALID_ARG;
    eval_terms(*in, *out);
    return CREDIT_OK;
}

credit_status credit_load_model(const char *path) {
    if (!path) return CREDIT_ERR_INVALID_ARG;
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    Calib c;
    if (!read_calib(path, c)) return CREDIT_ERR_IO;
    c.mlp_dir = dir_of(path);
    finish_calib(*device_info(dev), c);
    {
        std::lock_guard<std::mutex> lk(g_cal_mu);
        g_cal[dev] = c;
    }
    bump_plan_generation();
    if (!c.mlp_path.empty()) {
        std::string p = c.mlp_path;
        if (p[0] != '/') p = dir_of(path) + p;  // relative to the calibration file
        if (credit_mlp_load(p.c_str()) != CREDIT_OK) return CREDIT_ERR_IO;
    }
    return CREDIT_OK;
}

credit_status credit_calibrate(const char *path, int64_t max_bytes) {
    if (!path) return CREDIT_ERR_INVALID_ARG;
    if (max_bytes <= 0) max_bytes = 4LL << 30;
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    const DeviceInfo &di = *device_info(dev);
    Calib c;
    if ((st = credit_microbench(&c.mb, 15)) != CREDIT_OK) return st;
    {
        const char *e = std::getenv("CREDIT_HBM_GBS");
        c.hbm_gbs = e ? std::atof(e) : 0.0;
    }
    // buffers for the baseline timings
    const long long half = max_bytes / 2;
    void *in = nullptr, *out = nullptr;
    float *gb = nullptr, *sc = nullptr;
    const long long max_cols = 1LL << 20, max_rows = 1LL << 16;
    if (cudaMalloc(&in, half) != cudaSuccess || cudaMalloc(&out, half) != cudaSuccess ||
        cudaMalloc(&gb, 2 * max_cols * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&sc, 2 * max_rows * sizeof(float)) != cudaSuccess) {
        cudaFree(in);
        cudaFree(out);
        cudaFree(gb);
        cudaFree(sc);
        return CREDIT_ERR_CUDA;
    }
    // finite values everywhere: bytes 0x3c give small positive numbers in every format
    cudaMemset(in, 0x3c, half);
    cudaMemset(gb, 0, 2 * max_cols * sizeof(float));
    cudaMemset(sc, 0x3c, 2 * max_rows * sizeof(float));
    cudaEvent_t a0, a1;
    cudaEventCreate(&a0);
    cudaEventCreate(&a1);
    const long long Rs[6] = {64, 256, 1024, 4096, 16384, 65536};
    const long long Cs[6] = {1024, 4096, 16384, 65536, 262144, 1048576};
    cudaError_t err = cudaSuccess;
    for (int op = 0; op < 4 && err == cudaSuccess; ++op) {
        for (int dt = 0; dt < 3 && err == cudaSuccess; ++dt) {
            const int tout = op == 1 ? 0 : dt;
            for (long long R : Rs)
                for (long long Cn : Cs) {
                    const long long bytes_in = R * Cn * dtype_size(dt);
                    const long long bytes_out = op == 1 ? R * 4 : R * Cn * dtype_size(tout);
                    if (bytes_in > half || bytes_out > half) continue;
                    credit_plan_t p;
                    baseline_plan(di, dev, op, R, Cn, dt, tout, &p);
                    credit_args a;
                    std::memset(&a, 0, sizeof(a));
                    a.op = op;
                    a.in = in;
                    a.out = out;
                    a.rows = R;
                    a.cols = Cn;
                    a.in_dtype = dt;
                    a.out_dtype = tout;
                    a.in_scale = sc;
                    a.out_scale = sc + max_rows;
                    a.gamma = (op >= 2) ? gb : nullptr;
                    a.beta = (op == 2) ? gb + max_cols : nullptr;
                    a.eps = -1.0f;
                    std::vector<float> v;
                    for (int k = 0; k < 9; ++k) {
                        cudaEventRecord(a0);
                        if (credit_run_ex(&a, &p, nullptr) != CREDIT_OK) {
                            err = cudaErrorUnknown;
                            break;
                        }
                        cudaEventRecord(a1);
                        cudaEventSynchronize(a1);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, a0, a1);
                        if (k >= 2) v.push_back(ms * 1e3f);
                    }
                    if (err != cudaSuccess) break;
                    std::sort(v.begin(), v.end());
                    c.tb[tb_key(op, dt)].push_back({R, Cn, v[v.size() / 2], 0.0});
                }
        }
    }
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    cudaFree(in);
    cudaFree(out);
    cudaFree(gb);
    cudaFree(sc);
    if (err != cudaSuccess) return CREDIT_ERR_CUDA;
    // control kernel: excess of P over P = 1 with the same launch shape
    const long long CR[5] = {64, 1024, 4096, 16384, 65536};
    for (int dt = 0; dt < 3; ++dt)
        for (long long Cn : Cs)
            for (long long R : CR) {
                for (int P : kPs) {
                    float up = 0, u1 = 0;
                    if (credit_control_time(CREDIT_OP_SOFTMAX, R, Cn, static_cast<credit_dtype>(dt), P, 7, &up) !=
                        CREDIT_OK)
                        continue;
                    // the one-CTA control keeps P's dynamic shared memory footprint: rows of N / P elements
                    if (credit_control_time(CREDIT_OP_SOFTMAX, R, (Cn + P - 1) / P, static_cast<credit_dtype>(dt), 1,
                                            7, &u1) != CREDIT_OK)
                        continue;
                    c.ctrl[dt].push_back({R, Cn, P, up, u1});
                }
            }
    finish_calib(di, c);
    {  // a learned model named by the calibration loaded before stays named by the new one: by the same
       // relative name in the same directory, else by its path from the old file's directory
        std::lock_guard<std::mutex> lk(g_cal_mu);
        if (g_cal[dev].loaded && !g_cal[dev].mlp_path.empty()) {
            const Calib &o = g_cal[dev];
            if (o.mlp_path[0] == '/' || same_dir(o.mlp_dir, dir_of(path))) c.mlp_path = o.mlp_path;
            else c.mlp_path = absolute(o.mlp_dir + o.mlp_path);
        }
    }
    if (!write_calib(path, c, di)) return CREDIT_ERR_IO;
    {
        std::lock_guard<std::mutex> lk(g_cal_mu);
        g_cal[dev] = c;
    }
    bump_plan_generation();
    return CREDIT_OK;
}

}  // extern "C"
