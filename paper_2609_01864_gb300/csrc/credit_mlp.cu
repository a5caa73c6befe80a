// credit_mlp.cu -- learned latency model: a 3 x 64 MLP trained on the GPU
// with hand-written FP32 kernels (no tensor cores: the matrices are 64 wide).
//
// Input: kIn features of one (shape, dtype, op, candidate plan) (see
// credit_mlp_features).  Output: predicted log2 of the latency in us.  An
// ensemble of independently initialised members predicts the mean of their
// outputs (lower variance than one network, which matters when candidates
// differ by a few percent).
// Training: minibatch Adam on the mean squared error of standardised
// targets; features and targets are standardised with the training set's
// mean / standard deviation, kept with the weights.
// Planning: the argmin of the predicted latency over the legal candidates
// (one-CTA, cluster P in {2, 4, 8, 16}, two-pass with G in {1, 2, 4, 8} and
// the split factor); single planning queries run the same network on the host, batched
// evaluation runs the inference kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <mutex>
#include <numeric>
#include <random>
#include <vector>

#include "credit_model.h"
#include "credit_rows.cuh"

namespace credit {

namespace {

constexpr int kIn = 21, kH = 64;
// fill candidates of cluster plans that leave SMs idle (share of the rows)
constexpr float kFillShares[] = {0.15f, 0.2f, 0.3f, 0.4f};
// Predictions closer than this (log2 of the latency ratio, 0.7%) are below the ensemble's resolution: among
// them the planner takes a plan without a fill (one launch instead of three, no shared-HBM contention).
constexpr float kFillTieLog2 = 0.01f;
constexpr int kFillMinIdle = 16;
constexpr long long kFillMinRows = 64;
// flat layout: W1 (64 x kIn), b1, W2 (64x64), b2, W3 (64x64), b3, W4 (1x64), b4
constexpr int kOffW[4] = {0, kH * kIn + kH, kH * kIn + kH + kH * kH + kH, kH * kIn + kH + 2 * (kH * kH + kH)};
constexpr int kFanIn[4] = {kIn, kH, kH, kH};
constexpr int kFanOut[4] = {kH, kH, kH, 1};
constexpr int kParams = kH * kIn + kH + 2 * (kH * kH + kH) + kH + 1;

struct Model {
    bool loaded = false;
    std::vector<float> p;            // kParams
    float fmean[kIn], fstd[kIn];     // feature standardisation
    float tmean = 0.0f, tstd = 1.0f;  // target standardisation
};
std::vector<Model> g_models;  // the ensemble (empty: no learned model)
std::mutex g_mu;
constexpr int kMaxMembers = 16;

// ------------------------------------------------------------------ kernels
// out[s][u] = act(b[u] + sum_k W[u][k] in[s][k]); one thread per (s, u)
__global__ void k_fwd(const float *__restrict__ W, const float *__restrict__ b, const float *__restrict__ in,
                      float *__restrict__ out, int n, int fi, int fo, int relu) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(n) * fo) return;
    const int s = static_cast<int>(idx / fo), u = static_cast<int>(idx % fo);
    float acc = b[u];
    const float *w = W + static_cast<long long>(u) * fi, *x = in + static_cast<long long>(s) * fi;
    for (int k = 0; k < fi; ++k) acc = fmaf(w[k], x[k], acc);
    out[idx] = relu ? fmaxf(acc, 0.0f) : acc;
}

// dy[s] = 2 (y[s] - t[s]) / n
__global__ void k_out_delta(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) dy[s] = 2.0f * (y[s] - t[s]) / static_cast<float>(n);
}

// din[s][k] = (sum_u W[u][k] dout[s][u]) * (act[s][k] > 0); one thread per (s, k)
__global__ void k_bwd_delta(const float *__restrict__ W, const float *__restrict__ dout, const float *__restrict__ act,
                            float *__restrict__ din, int n, int fi, int fo) {
    const long long idx = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= static_cast<long long>(n) * fi) return;
    const int s = static_cast<int>(idx / fi), k = static_cast<int>(idx % fi);
    float acc = 0.0f;
    for (int u = 0; u < fo; ++u) acc = fmaf(W[static_cast<long long>(u) * fi + k], dout[static_cast<long long>(s) * fo + u], acc);
    din[idx] = act[idx] > 0.0f ? acc : 0.0f;
}

// gW[u][k] = sum_s dout[s][u] in[s][k], gb[u] = sum_s dout[s][u]; one thread
// per weight (k == fi: the bias), summed in sample order (deterministic)
__global__ void k_grad(const float *__restrict__ dout, const float *__restrict__ in, float *__restrict__ gW,
                       float *__restrict__ gb, int n, int fi, int fo) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= fo * (fi + 1)) return;
    const int u = idx / (fi + 1), k = idx % (fi + 1);
    float acc = 0.0f;
    if (k == fi) {
        for (int s = 0; s < n; ++s) acc += dout[static_cast<long long>(s) * fo + u];
        gb[u] = acc;
    } else {
        for (int s = 0; s < n; ++s)
            acc = fmaf(dout[static_cast<long long>(s) * fo + u], in[static_cast<long long>(s) * fi + k], acc);
        gW[u * fi + k] = acc;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// sum of squared errors into out[0] (one block)
__global__ void k_sse(const float *__restrict__ y, const float *__restrict__ t, int n, float *out) {
    __shared__ float red[33];
    float acc = 0.0f;
    for (int s = threadIdx.x; s < n; s += blockDim.x) {
        const float d = y[s] - t[s];
        acc = fmaf(d, d, acc);
    }
    const float r = block_allreduce<false>(acc, red);
    if (threadIdx.x == 0) out[0] = r;
}

inline unsigned blocks(long long n, int t) { return static_cast<unsigned>((n + t - 1) / t); }

// Device workspace for one batch size.
struct Dev {
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float *x = nullptr, *t = nullptr, *a[4] = {nullptr, nullptr, nullptr, nullptr}, *y = nullptr;
    float *d[4] = {nullptr, nullptr, nullptr, nullptr}, *dy = nullptr, *loss = nullptr;
    int cap = 0;
    bool alloc(int n) {
        cap = n;
        bool ok = cudaMalloc(&p, kParams * 4) == cudaSuccess && cudaMalloc(&g, kParams * 4) == cudaSuccess &&
                  cudaMalloc(&m, kParams * 4) == cudaSuccess && cudaMalloc(&v, kParams * 4) == cudaSuccess &&
                  cudaMalloc(&x, static_cast<size_t>(n) * kIn * 4) == cudaSuccess &&
                  cudaMalloc(&t, static_cast<size_t>(n) * 4) == cudaSuccess &&
                  cudaMalloc(&y, static_cast<size_t>(n) * 4) == cudaSuccess &&
                  cudaMalloc(&dy, static_cast<size_t>(n) * 4) == cudaSuccess && cudaMalloc(&loss, 16) == cudaSuccess;
        for (int l = 0; l < 3 && ok; ++l)
            ok = cudaMalloc(&a[l], static_cast<size_t>(n) * kH * 4) == cudaSuccess &&
                 cudaMalloc(&d[l], static_cast<size_t>(n) * kH * 4) == cudaSuccess;
        if (ok) {
            cudaMemset(m, 0, kParams * 4);
            cudaMemset(v, 0, kParams * 4);
        }
        return ok;
    }
    void release() {
        float *all[] = {p, g, m, v, x, t, y, dy, loss, a[0], a[1], a[2], d[0], d[1], d[2]};
        for (float *q : all) cudaFree(q);
    }
    // forward: x -> a[0..2] -> y
    void forward(int n) {
        const float *in = x;
        for (int l = 0; l < 4; ++l) {
            const float *W = p + kOffW[l], *b = W + kFanOut[l] * kFanIn[l];
            float *out = l < 3 ? a[l] : y;
            k_fwd<<<blocks(static_cast<long long>(n) * kFanOut[l], 256), 256>>>(W, b, in, out, n, kFanIn[l],
                                                                                kFanOut[l], l < 3);
            in = out;
        }
    }
    // Adam step number `step` (1, 2, ...) on p from g, with the moments m, v
    void adam(int step, float lr) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.0f - std::pow(b1, static_cast<float>(step));
        const float c2 = 1.0f - std::pow(b2, static_cast<float>(step));
        k_adam<<<blocks(kParams, 256), 256>>>(p, g, m, v, kParams, lr, b1, b2, eps, c1, c2);
    }
    // backward into g (forward must have run on the same batch)
    void backward(int n) {
        k_out_delta<<<blocks(n, 256), 256>>>(y, t, dy, n);
        const float *dout = dy;
        for (int l = 3; l >= 0; --l) {
            const float *in = l == 0 ? x : a[l - 1];
            float *gW = g + kOffW[l], *gb = gW + kFanOut[l] * kFanIn[l];
            k_grad<<<blocks(kFanOut[l] * (kFanIn[l] + 1), 128), 128>>>(dout, in, gW, gb, n, kFanIn[l], kFanOut[l]);
            if (l > 0) {
                const float *W = p + kOffW[l];
                k_bwd_delta<<<blocks(static_cast<long long>(n) * kFanIn[l], 256), 256>>>(W, dout, a[l - 1], d[l - 1],
                                                                                         n, kFanIn[l], kFanOut[l]);
                dout = d[l - 1];
            }
        }
    }
};

void host_forward(const Model &mdl, const float *xin, float *yout_log2us) {
    float x[kIn], h[kH], h2[kH];
    for (int k = 0; k < kIn; ++k) x[k] = (xin[k] - mdl.fmean[k]) / mdl.fstd[k];
    const float *in = x;
    int fi = kIn;
    for (int l = 0; l < 3; ++l) {
        const float *W = mdl.p.data() + kOffW[l], *b = W + kH * fi;
        for (int u = 0; u < kH; ++u) {
            float acc = b[u];
            for (int k = 0; k < fi; ++k) acc = fmaf(W[u * fi + k], in[k], acc);
            (l % 2 ? h2 : h)[u] = acc > 0.0f ? acc : 0.0f;
        }
        in = l % 2 ? h2 : h;
        fi = kH;
    }
    const float *W = mdl.p.data() + kOffW[3];
    float acc = W[kH];
    for (int k = 0; k < kH; ++k) acc = fmaf(W[k], in[k], acc);
    *yout_log2us = acc * mdl.tstd + mdl.tmean;
}

}  // namespace

// Features of one candidate: log2 rows, log2 cols, input dtype one-hot (3),
// op one-hot (4), path one-hot (one-CTA, two-pass, cluster), log2 P, log2 G,
// log2 of the algorithmic bytes, output bytes per element, log2 of the input
// bytes one CTA handles, log2 of the CTAs per SM (152 SMs) the rows need,
// tensor-memory retention (0 / 1), and the share of rows given to the fill.
void mlp_features(int op, int tin, int tout, long long rows, long long cols, int path, int P, int G, int retain_tm,
                  float fill, float *f) {
    std::memset(f, 0, kIn * sizeof(float));
    f[0] = std::log2(static_cast<float>(rows));
    f[1] = std::log2(static_cast<float>(cols));
    f[2 + tin] = 1.0f;
    f[5 + op] = 1.0f;
    f[9 + (path == CREDIT_PATH_ONE_CTA ? 0 : path == CREDIT_PATH_TWO_PASS ? 1 : 2)] = 1.0f;
    f[12] = std::log2(static_cast<float>(P < 1 ? 1 : P));
    f[13] = std::log2(static_cast<float>(G < 1 ? 1 : G));
    const double ob = op == 1 ? 0.0 : dtype_size(tout);
    const double bytes = static_cast<double>(rows) * cols * (dtype_size(tin) + ob) + (op == 1 ? rows * 4.0 : 0.0);
    f[14] = static_cast<float>(std::log2(bytes));
    f[15] = static_cast<float>(ob);
    const int split = path == CREDIT_PATH_TWO_PASS ? (G < 1 ? 1 : G) : (P < 1 ? 1 : P);
    f[16] = static_cast<float>(std::log2(static_cast<double>(cols) * dtype_size(tin) / split + 1.0));
    f[17] = static_cast<float>(std::log2(static_cast<double>(rows) * split / 152.0));
    f[18] = retain_tm ? 1.0f : 0.0f;
    f[19] = fill;
    // contiguous rows all start on the 16-byte grid: the staged kernels then keep gamma / beta in shared
    // memory and use whole 16-byte groups from each row's first element
    f[20] = (cols * dtype_size(tin)) % 16 == 0 ? 1.0f : 0.0f;
}

static bool learned_plan_impl(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin,
                              int tout, bool allow_cluster, credit_plan_t *p);

bool learned_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                  credit_plan_t *p) {
    return learned_plan_impl(di, device, op, rows, cols, tin, tout, true, p);
}

bool learned_plan_no_cluster(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin,
                             int tout, credit_plan_t *p) {
    return learned_plan_impl(di, device, op, rows, cols, tin, tout, false, p);
}

static bool learned_plan_impl(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin,
                              int tout, bool allow_cluster, credit_plan_t *p) {
    std::vector<Model> ens;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_models.empty()) return false;
        ens = g_models;
    }
    std::vector<std::pair<float, credit_plan_t>> cands;  // (mean predicted log2 latency, plan), in order
    auto consider = [&](int path, int P, int G, long long smem, int retain, float fill) {
        float f[kIn], y = 0.0f;
        mlp_features(op, tin, tout, rows, cols, path, P, G, retain == CREDIT_RETAIN_TMEM, fill, f);
        for (const Model &m : ens) {
            float ym;
            host_forward(m, f, &ym);
            y += ym;
        }
        y /= static_cast<float>(ens.size());
        credit_plan_t c{};
        c.path = path;
        c.cluster_size = path == CREDIT_PATH_TWO_PASS ? 1 : P;
        c.ctas_per_row = path == CREDIT_PATH_TWO_PASS ? G : P;
        c.smem_bytes = smem;
        c.retain = retain;
        c.fill_share = fill;
        c.predicted_us = std::exp2(y);
        c.source = 1;
        cands.emplace_back(y, c);
    };
    const int isz = dtype_size(tin);
    for (int P : {1, 2, 4, 8, 16}) {
        if (op == 1 && P == 1) continue;
        if (P > 1 && !allow_cluster) continue;
        const int path = P == 1 ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
        // a cluster plan that leaves >= kFillMinIdle SMs idle also comes with a
        // fill of the last rows by the split two-pass path on those SMs
        auto with_fills = [&](long long smem, int retain, int maxc) {
            consider(path, P, P, smem, retain, 0.0f);
            if (P > 1 && rows >= kFillMinRows && di.sm_count - P * maxc >= kFillMinIdle)
                for (float f : kFillShares) consider(path, P, P, smem, retain, f);
        };
        RingCfg rc;
        int maxc = 0;
        if (ring_config(di, cols, isz, P, 0, 0, 0, 0, 0, &rc) &&
            (maxc = ring_max_clusters(device, op, tin, tout, P, rc.threads, rc.smem)) > 0)
            with_fills(rc.smem, CREDIT_RETAIN_SMEM, maxc);
        const bool tm_op = op != 1 && !(tout == 2 && (op == 2 || op == 3));
        if (tm_op && ring_config_tm(di, cols, isz, P, 0, 0, 0, &rc) &&
            (maxc = ring_max_clusters(device, op, tin, tout, P, rc.threads, rc.smem, true)) > 0)
            with_fills(rc.smem, CREDIT_RETAIN_TMEM, maxc);
    }
    // two-pass: G in {1, 2, 4, 8} with >= 1024 16-byte groups per CTA, and the split rule's G
    const long long groups = cols * isz / 16;
    for (int G : {1, 2, 4, 8})
        if (G == 1 || groups / G >= 1024) consider(CREDIT_PATH_TWO_PASS, 1, G, 0, CREDIT_RETAIN_AUTO, 0.0f);
    const int Gs = two_pass_split(di.sm_count, rows, cols, isz);
    if (Gs > 1 && Gs != 2 && Gs != 4 && Gs != 8) consider(CREDIT_PATH_TWO_PASS, 1, Gs, 0, CREDIT_RETAIN_AUTO, 0.0f);
    if (cands.empty()) return false;
    float best = 1e30f;
    for (const auto &c : cands) best = std::min(best, c.first);
    // the lowest prediction; within kFillTieLog2 of it, the lowest one without a fill
    int pick = -1, pick_nofill = -1;
    for (int i = 0; i < static_cast<int>(cands.size()); ++i) {
        const float y = cands[i].first;
        if (pick < 0 && y == best) pick = i;
        if (cands[i].second.fill_share == 0.0f && y <= best + kFillTieLog2 &&
            (pick_nofill < 0 || y < cands[pick_nofill].first))
            pick_nofill = i;
    }
    if (pick_nofill >= 0) pick = pick_nofill;
    best = cands[pick].first;
    credit_plan_t bp = cands[pick].second;
    // predicted latency anchored on the measured baseline: T_B (calibration, Eq. 7) times the model's ratio of
    // the pick to the baseline plan (the ratio is what the network learns; its per-shape level cancels)
    credit_plan_t base;
    double T_B = 0.0;
    if (baseline_estimate(di, device, op, rows, cols, tin, tout, &base, &T_B) && T_B > 0.0) {
        float fb[kIn], yb = 0.0f;
        mlp_features(op, tin, tout, rows, cols, base.path, base.cluster_size, base.ctas_per_row,
                     base.retain == CREDIT_RETAIN_TMEM, 0.0f, fb);
        for (const Model &m : ens) {
            float ym;
            host_forward(m, fb, &ym);
            yb += ym;
        }
        yb /= static_cast<float>(ens.size());
        bp.predicted_us = static_cast<float>(T_B * std::exp2(static_cast<double>(best) - yb));
    }
    *p = bp;
    return true;
}

}  // namespace credit

using namespace credit;

extern "C" {

int64_t credit_mlp_num_params(void) { return kParams; }

credit_status credit_mlp_features(int32_t op, int32_t in_dtype, int32_t out_dtype, int64_t rows, int64_t cols,
                                  int32_t path, int32_t P, int32_t G, int32_t retain, float fill_share, float *out) {
    if (!out || op < 0 || op > 3 || in_dtype < 0 || in_dtype > 2 || out_dtype < 0 || out_dtype > 2 || rows <= 0 ||
        cols <= 0 || path < 0 || path > 2 || retain < 0 || retain > 2 || !(fill_share >= 0.0f && fill_share <= 1.0f))
        return CREDIT_ERR_INVALID_ARG;
    mlp_features(op, in_dtype, op == 1 ? 0 : out_dtype, rows, cols, path, P, G,
                 path != CREDIT_PATH_TWO_PASS && retain == CREDIT_RETAIN_TMEM,
                 path == CREDIT_PATH_CLUSTER ? fill_share : 0.0f, out);
    return CREDIT_OK;
}

// One forward + backward on the GPU with explicit parameters and raw
// (unstandardised) inputs: the MSE loss and its gradient (for checking the
// kernels against an FP64 reference).  Host arrays.
credit_status credit_mlp_grad(const float *params, const float *X, const float *t, int64_t n, float *grad,
                              float *loss) {
    if (!params || !X || !t || !grad || !loss || n <= 0 || n > (1 << 20)) return CREDIT_ERR_INVALID_ARG;
    Dev d;
    if (!d.alloc(static_cast<int>(n))) {
        d.release();
        return CREDIT_ERR_CUDA;
    }
    cudaMemcpy(d.p, params, kParams * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d.x, X, n * kIn * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d.t, t, n * 4, cudaMemcpyHostToDevice);
    d.forward(static_cast<int>(n));
    d.backward(static_cast<int>(n));
    k_sse<<<1, 256>>>(d.y, d.t, static_cast<int>(n), d.loss);
    float sse = 0.0f;
    cudaError_t e = cudaMemcpy(grad, d.g, kParams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&sse, d.loss, 4, cudaMemcpyDeviceToHost);
    d.release();
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    *loss = sse / static_cast<float>(n);
    return CREDIT_OK;
}

// One Adam step of the training kernel on host arrays (params, m, v updated
// in place from grad), for checking the kernel against an FP64 reference.
credit_status credit_mlp_adam_step(float *params, const float *grad, float *m, float *v, int32_t step, float lr) {
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.0f)) return CREDIT_ERR_INVALID_ARG;
    Dev d;
    if (!d.alloc(1)) {
        d.release();
        return CREDIT_ERR_CUDA;
    }
    cudaMemcpy(d.p, params, kParams * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d.g, grad, kParams * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d.m, m, kParams * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(d.v, v, kParams * 4, cudaMemcpyHostToDevice);
    d.adam(step, lr);
    cudaError_t e = cudaMemcpy(params, d.p, kParams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(m, d.m, kParams * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(v, d.v, kParams * 4, cudaMemcpyDeviceToHost);
    d.release();
    return e == cudaSuccess ? CREDIT_OK : CREDIT_ERR_CUDA;
}
}  // extern "C"

namespace credit {
namespace {
// Train one member from scratch (see credit_mlp_train); the model is returned
// in *out, not installed.
credit_status train_one(const float *X, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                        uint64_t seed, float *loss_curve, Model *out) {
    Model mdl;
    // standardisation
    for (int k = 0; k < kIn; ++k) {
        double s = 0, s2 = 0;
        for (int64_t i = 0; i < n; ++i) s += X[i * kIn + k];
        const double mu = s / n;
        for (int64_t i = 0; i < n; ++i) s2 += (X[i * kIn + k] - mu) * (X[i * kIn + k] - mu);
        const double sd = std::sqrt(s2 / n);
        mdl.fmean[k] = static_cast<float>(mu);
        mdl.fstd[k] = sd > 1e-6 ? static_cast<float>(sd) : 1.0f;
    }
    {
        double s = 0, s2 = 0;
        for (int64_t i = 0; i < n; ++i) s += y[i];
        const double mu = s / n;
        for (int64_t i = 0; i < n; ++i) s2 += (y[i] - mu) * (y[i] - mu);
        mdl.tmean = static_cast<float>(mu);
        mdl.tstd = static_cast<float>(std::max(1e-6, std::sqrt(s2 / n)));
    }
    std::vector<float> Xs(n * kIn), ys(n);
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < kIn; ++k) Xs[i * kIn + k] = (X[i * kIn + k] - mdl.fmean[k]) / mdl.fstd[k];
        ys[i] = (y[i] - mdl.tmean) / mdl.tstd;
    }
    // He initialisation
    std::mt19937_64 rng(seed);
    mdl.p.assign(kParams, 0.0f);
    for (int l = 0; l < 4; ++l) {
        std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / kFanIn[l]));
        for (int i = 0; i < kFanOut[l] * kFanIn[l]; ++i) mdl.p[kOffW[l] + i] = nd(rng);
    }
    const int B = static_cast<int>(std::min<int64_t>(batch, n));
    Dev d;
    if (!d.alloc(B)) {
        d.release();
        return CREDIT_ERR_CUDA;
    }
    cudaMemcpy(d.p, mdl.p.data(), kParams * 4, cudaMemcpyHostToDevice);
    std::vector<int64_t> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    std::vector<float> bx(static_cast<size_t>(B) * kIn), bt(B);
    int step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        double ep_loss = 0.0;
        int nb = 0;
        for (int64_t s0 = 0; s0 + B <= n; s0 += B) {
            for (int i = 0; i < B; ++i) {
                std::memcpy(&bx[static_cast<size_t>(i) * kIn], &Xs[perm[s0 + i] * kIn], kIn * 4);
                bt[i] = ys[perm[s0 + i]];
            }
            cudaMemcpy(d.x, bx.data(), bx.size() * 4, cudaMemcpyHostToDevice);
            cudaMemcpy(d.t, bt.data(), bt.size() * 4, cudaMemcpyHostToDevice);
            d.forward(B);
            d.backward(B);
            d.adam(++step, lr);
            if (loss_curve) {
                k_sse<<<1, 256>>>(d.y, d.t, B, d.loss);
                float sse = 0;
                cudaMemcpy(&sse, d.loss, 4, cudaMemcpyDeviceToHost);
                ep_loss += sse / B;
                ++nb;
            }
        }
        if (loss_curve) loss_curve[ep] = nb ? static_cast<float>(ep_loss / nb) : 0.0f;
    }
    cudaError_t e = cudaMemcpy(mdl.p.data(), d.p, kParams * 4, cudaMemcpyDeviceToHost);
    d.release();
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    mdl.loaded = true;
    *out = mdl;
    return CREDIT_OK;
}
}  // namespace
}  // namespace credit

extern "C" {

credit_status credit_mlp_train(const float *X, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                               uint64_t seed, float *loss_curve) {
    return credit_mlp_train_ensemble(X, y, n, 1, epochs, batch, lr, seed, loss_curve);
}

credit_status credit_mlp_train_ensemble(const float *X, const float *y, int64_t n, int32_t members, int32_t epochs,
                                        int32_t batch, float lr, uint64_t seed, float *loss_curve) {
    if (!X || !y || n < 2 || epochs < 1 || batch < 1 || members < 1 || members > kMaxMembers)
        return CREDIT_ERR_INVALID_ARG;
    std::vector<Model> ens(static_cast<size_t>(members));
    for (int m = 0; m < members; ++m) {
        const credit_status st = train_one(X, y, n, epochs, batch, lr, seed + static_cast<uint64_t>(m),
                                           m == 0 ? loss_curve : nullptr, &ens[static_cast<size_t>(m)]);
        if (st != CREDIT_OK) return st;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_models = ens;
    }
    bump_plan_generation();
    return CREDIT_OK;
}

int32_t credit_mlp_members(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    return static_cast<int32_t>(g_models.size());
}

// Batched inference on the GPU: predicted log2 us for n feature rows.
credit_status credit_mlp_predict(const float *X, int64_t n, float *out) {
    if (!X || !out || n <= 0 || n > (1 << 22)) return CREDIT_ERR_INVALID_ARG;
    std::vector<Model> ens;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_models.empty()) return CREDIT_ERR_NOT_INITIALIZED;
        ens = g_models;
    }
    Dev d;
    if (!d.alloc(static_cast<int>(n))) {
        d.release();
        return CREDIT_ERR_CUDA;
    }
    std::vector<float> Xs(n * kIn), ym(n);
    for (int64_t i = 0; i < n; ++i) out[i] = 0.0f;
    cudaError_t e = cudaSuccess;
    for (const Model &mdl : ens) {
        for (int64_t i = 0; i < n; ++i)
            for (int k = 0; k < kIn; ++k) Xs[i * kIn + k] = (X[i * kIn + k] - mdl.fmean[k]) / mdl.fstd[k];
        cudaMemcpy(d.p, mdl.p.data(), kParams * 4, cudaMemcpyHostToDevice);
        cudaMemcpy(d.x, Xs.data(), Xs.size() * 4, cudaMemcpyHostToDevice);
        d.forward(static_cast<int>(n));
        if ((e = cudaMemcpy(ym.data(), d.y, n * 4, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
        for (int64_t i = 0; i < n; ++i) out[i] += ym[i] * mdl.tstd + mdl.tmean;
    }
    d.release();
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    for (int64_t i = 0; i < n; ++i) out[i] /= static_cast<float>(ens.size());
    return CREDIT_OK;
}

credit_status credit_mlp_save(const char *path) {
    std::vector<Model> ens;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_models.empty()) return CREDIT_ERR_NOT_INITIALIZED;
        ens = g_models;
    }
    FILE *f = path ? std::fopen(path, "w") : nullptr;
    if (!f) return CREDIT_ERR_IO;
    // version 2: the member count, then every member (standardisation, parameters)
    std::fprintf(f, "credit-mlp 2 %d %d %d %d\n", kIn, kH, kParams, static_cast<int>(ens.size()));
    for (const Model &mdl : ens) {
        for (int k = 0; k < kIn; ++k) std::fprintf(f, "%.9g %.9g\n", mdl.fmean[k], mdl.fstd[k]);
        std::fprintf(f, "%.9g %.9g\n", mdl.tmean, mdl.tstd);
        for (int i = 0; i < kParams; ++i) std::fprintf(f, "%.9g\n", mdl.p[i]);
    }
    return std::fclose(f) == 0 ? CREDIT_OK : CREDIT_ERR_IO;
}

// Reads version 1 (one network) and version 2 (an ensemble).
credit_status credit_mlp_load(const char *path) {
    FILE *f = path ? std::fopen(path, "r") : nullptr;
    if (!f) return CREDIT_ERR_IO;
    int a = 0, b = 0, c = 0, v = 0, members = 1;
    bool ok = std::fscanf(f, "credit-mlp %d %d %d %d", &v, &a, &b, &c) == 4 && a == kIn && b == kH && c == kParams &&
              (v == 1 || v == 2);
    if (ok && v == 2) ok = std::fscanf(f, "%d", &members) == 1 && members >= 1 && members <= kMaxMembers;
    std::vector<Model> ens(ok ? static_cast<size_t>(members) : 0);
    for (Model &mdl : ens) {
        for (int k = 0; ok && k < kIn; ++k) ok = std::fscanf(f, "%f %f", &mdl.fmean[k], &mdl.fstd[k]) == 2;
        if (ok) ok = std::fscanf(f, "%f %f", &mdl.tmean, &mdl.tstd) == 2;
        mdl.p.resize(kParams);
        for (int i = 0; ok && i < kParams; ++i) ok = std::fscanf(f, "%f", &mdl.p[i]) == 1;
        mdl.loaded = ok;
    }
    std::fclose(f);
    if (!ok) return CREDIT_ERR_IO;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_models = ens;
    }
    bump_plan_generation();
    return CREDIT_OK;
}

}  // extern "C"
