// credit_plan.cpp -- plan selection (CREDIT Sec. III-D).
//
// Candidates for a shape: the one-CTA staged path (P = 1), the cluster path
// for every P in {2, 4, 8, 16} that passes the capacity check of Eq. 3 and
// can be scheduled (max active clusters > 0), and the two-pass global-reread
// path.  Without calibration data the built-in heuristic below is used; the
// analytic model of Eq. 7-9 and the learned model plug in through
// credit_model.cpp.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <unordered_map>

#include "credit_host.h"
#include "credit_model.h"

namespace credit {

// Plans chosen by credit_plan_ex, per (device, op, rows, cols, dtypes): the
// learned planner evaluates every candidate through the network ensemble on
// the host, which costs more than a short launch, so a call without a plan
// reuses the choice made for the same shape.  Emptied when the calibration or
// the model changes; bypassed while CREDIT_FORCE_PATH or CREDIT_MODEL select
// a planner by environment.
namespace {
struct PlanKey {
    int dev, op, tin, tout;
    long long rows, cols;
    bool operator==(const PlanKey &o) const {
        return dev == o.dev && op == o.op && tin == o.tin && tout == o.tout && rows == o.rows && cols == o.cols;
    }
};
struct PlanKeyHash {
    size_t operator()(const PlanKey &k) const {
        uint64_t h = 1469598103934665603ull;
        const long long v[6] = {k.dev, k.op, k.tin, k.tout, k.rows, k.cols};
        for (long long x : v) h = (h ^ static_cast<uint64_t>(x)) * 1099511628211ull;
        return static_cast<size_t>(h);
    }
};
std::mutex g_plan_mu;
std::unordered_map<PlanKey, credit_plan_t, PlanKeyHash> g_plan_cache;
std::atomic<unsigned long long> g_plan_gen{0};
unsigned long long g_cache_gen = 0;
constexpr size_t kPlanCacheMax = 4096;
}  // namespace

void bump_plan_generation() { g_plan_gen.fetch_add(1); }

static bool env_force(const DeviceInfo *di, credit_plan_t *p, long long cols, int tin) {
    const char *fp = std::getenv("CREDIT_FORCE_PATH");
    if (!fp || !*fp) return false;
    std::memset(p, 0, sizeof(*p));
    const char *fP = std::getenv("CREDIT_FORCE_P");
    const char *fG = std::getenv("CREDIT_FORCE_G");
    const char *fT = std::getenv("CREDIT_FORCE_THREADS");
    const char *fR = std::getenv("CREDIT_FORCE_RING");
    const char *fC = std::getenv("CREDIT_FORCE_CHUNK");
    const char *fRd = std::getenv("CREDIT_FORCE_REDUCERS");
    p->threads = fT ? std::atoi(fT) : 0;
    p->ring_chunks = fR ? std::atoi(fR) : 0;
    p->chunk_bytes = fC ? std::atoi(fC) : 0;
    p->reducer_threads = fRd ? std::atoi(fRd) : 0;
    p->source = 2;
    if (!std::strcmp(fp, "one_cta") || !std::strcmp(fp, "cluster")) {
        const bool one = !std::strcmp(fp, "one_cta");
        p->path = one ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
        p->cluster_size = one ? 1 : (fP ? std::atoi(fP) : 4);
        p->ctas_per_row = p->cluster_size;
        RingCfg rc;
        if (di && ring_config(*di, cols, dtype_size(tin), p->cluster_size, p->ring_chunks, p->chunk_bytes,
                              p->threads, p->reducer_threads, 0, &rc))
            p->smem_bytes = rc.smem;
    } else if (!std::strcmp(fp, "two_pass")) {
        p->path = CREDIT_PATH_TWO_PASS;
        p->cluster_size = 1;
        p->ctas_per_row = fG ? std::atoi(fG) : 1;
    } else {
        return false;
    }
    return true;
}

// Split factor for the two-pass path: enough CTAs to cover the GPU several
// times over, but no CTA with fewer than ~1024 16-byte groups.
int two_pass_split(int sm_count, long long rows, long long cols, int isz) {
    const long long target = 4LL * sm_count;
    if (rows >= target) return 1;
    long long G = (target + rows - 1) / rows;
    const long long groups = (cols * isz) / 16;
    long long gmax = groups / 1024;
    if (gmax < 1) gmax = 1;
    if (G > gmax) G = gmax;
    if (G > 1024) G = 1024;
    return static_cast<int>(G < 1 ? 1 : G);
}

// Rule for int8 quantisation (measured on GB300, 4096 rows of 16K-256K FP32
// columns): the smallest cluster whose slices fit the tensor-memory tier
// (128 KiB); the fewest CTAs per row keeps the most rows in flight and the
// exchange shortest.  Two-pass when no staged plan fits.
static bool quant_plan(const DeviceInfo &di, int device, long long rows, long long cols, int tin, credit_plan_t *p) {
    const int isz = dtype_size(tin);
    for (int P : {1, 2, 4, 8, 16}) {
        RingCfg rc;
        if (!ring_config_tm(di, cols, isz, P, 0, 0, 0, &rc)) continue;
        if (ring_max_clusters(device, CREDIT_OP_QUANT_INT8, tin, CREDIT_INT8, P, rc.threads, rc.smem, true) <= 0) continue;
        p->path = P == 1 ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
        p->cluster_size = P;
        p->ctas_per_row = P;
        p->retain = CREDIT_RETAIN_TMEM;
        p->smem_bytes = rc.smem;
        return true;
    }
    p->path = CREDIT_PATH_TWO_PASS;
    p->cluster_size = 1;
    p->ctas_per_row = two_pass_split(di.sm_count, rows, cols, isz);
    return true;
}

void heuristic_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                    credit_plan_t *p) {
    std::memset(p, 0, sizeof(*p));
    p->source = 3;
    if (op == CREDIT_OP_QUANT_INT8 && quant_plan(di, device, rows, cols, tin, p)) return;
    const int isz = dtype_size(tin);
    if (op != 1) {
        // Smallest P whose slice is <= 64 KiB, else the smallest P that fits.
        int pick = 0;
        RingCfg best{};
        for (int pass = 0; pass < 2 && !pick; ++pass) {
            for (int P : {1, 2, 4, 8, 16}) {
                RingCfg rc;
                if (!ring_config(di, cols, isz, P, 0, 0, 0, 0, 0, &rc)) continue;
                if (pass == 0 && rc.body_max > 65536) continue;
                if (ring_max_clusters(device, op, tin, tout, P, rc.threads, rc.smem) <= 0) continue;
                pick = P;
                best = rc;
                break;
            }
        }
        if (pick) {
            p->path = pick == 1 ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
            p->cluster_size = pick;
            p->ctas_per_row = pick;
            p->smem_bytes = best.smem;
            return;
        }
    }
    p->path = CREDIT_PATH_TWO_PASS;
    p->cluster_size = 1;
    p->ctas_per_row = two_pass_split(di.sm_count, rows, cols, isz);
}

}  // namespace credit

using namespace credit;

extern "C" {

credit_status credit_plan_ex(credit_op op, int64_t rows, int64_t cols, credit_dtype in_dtype, credit_dtype out_dtype,
                             credit_plan_t *out) {
    const bool q8 = op == CREDIT_OP_QUANT_INT8;
    if (!out || ((op < 0 || op > 3) && !q8) || in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 3)
        return CREDIT_ERR_INVALID_ARG;
    if (q8 != (out_dtype == CREDIT_INT8)) return CREDIT_ERR_INVALID_ARG;
    if (q8 && in_dtype == CREDIT_FP8_E4M3) return CREDIT_ERR_UNSUPPORTED;
    if (rows < 0 || cols <= 0) return CREDIT_ERR_INVALID_ARG;
    const int tout = op == CREDIT_OP_LOGSUMEXP ? 0 : out_dtype;
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    const DeviceInfo *di = device_info(dev);
    if (!di) return CREDIT_ERR_NOT_INITIALIZED;
    if (env_force(di, out, cols, in_dtype)) return CREDIT_OK;
    const char *menv = std::getenv("CREDIT_MODEL");
    const bool cache = !(menv && *menv);
    const PlanKey key{dev, static_cast<int>(op), static_cast<int>(in_dtype), tout, rows, cols};
    const unsigned long long gen = g_plan_gen.load();
    if (cache) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        if (g_cache_gen != gen) {
            g_plan_cache.clear();
            g_cache_gen = gen;
        }
        const auto it = g_plan_cache.find(key);
        if (it != g_plan_cache.end()) {
            *out = it->second;
            return CREDIT_OK;
        }
    }
    // the calibration and the learned model cover the four ops of Sec. III-B; the quantiser takes the rule
    if (q8 || !model_plan(*di, dev, op, rows, cols, in_dtype, tout, out))
        heuristic_plan(*di, dev, op, rows, cols, in_dtype, tout, out);
    if (cache) {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        if (g_cache_gen == gen) {
            if (g_plan_cache.size() >= kPlanCacheMax) g_plan_cache.clear();
            g_plan_cache[key] = *out;
        }
    }
    return CREDIT_OK;
}

credit_status credit_plan(credit_op op, int64_t rows, int64_t cols, credit_dtype dtype, credit_plan_t *out) {
    return credit_plan_ex(op, rows, cols, dtype, op == CREDIT_OP_LOGSUMEXP ? CREDIT_F32 : dtype, out);
}

}  // extern "C"
