// credit_bwd.cu -- gradients of reduction-reuse row ops (the backward
// members of the workload suite, Sec. IV-A).
//
// Every row has two arrays, a and dy, and one stage (L = 1) of reductions
// followed by an elementwise pass over the same two arrays (Eq. 1).  With
// g = dy * gamma:
//   softmax    a = y, S0 = sum y dy                       dx = y (dy - S0)
//   layernorm  a = x, xh = (x - mean) rstd, S0 = sum g, S1 = sum g xh
//              dx = rstd (g - S0 / N - xh S1 / N)
//   rmsnorm    a = x, xh = x rstd, S1 = sum g xh          dx = rstd (g - xh S1 / N)
// (q = 1 or 2 plain sums); from logits z, with y = softmax(z) recomputed:
//   softmax    online (m, S = sum e^(z-m), T = sum e^(z-m) dy)
//              dz = e^(z-m) / S (dy - T / S)
//   xent       online (m, S), T = sum t (dy holds the targets t)
//              dz = w (e^(z-m) / S T - t)
// (q = 3, merged with rescaling); and of two-input statistics, with two
// outputs dx, dx2 and centred moments merged with Chan's formulas:
//   wvar       a = x, dy = w: (W, mu, M2), W = sum w, M2 = sum w (x - mu)^2
//              dx = g 2 w (x - mu) / W, dx2 = g ((x - mu)^2 - v) / W, v = M2 / W
//   pearson    a = x, dy = y: (n, xb, yb, Sxx, Syy, Sxy) centred co-moments
//              dx = g ((y - yb) / sqrt(Sxx Syy) - r (x - xb) / Sxx), dx2 symmetric
// (q = 3 or 6; each thread first sums about its own first elements, then
// converts once to the centred state before the merges).

// Paths:
//   k_bwd_staged   ONE_CTA (P = 1) and CLUSTER (P = 2..16).  A persistent
//                  cluster walks rows cl, cl + ncl, ...  Each CTA stages its
//                  slice of a and of dy (16-byte groups group_split(G, c, P)
//                  .. group_split(G, c + 1, P), Eq. 2) with bulk-async copies
//                  completed on an mbarrier, sums its partials, pushes them
//                  to every peer with st.async (completing on the peer's
//                  exchange mbarrier, Eq. 5-6), combines the P partials in
//                  the fixed order c = 0..P-1 (identical statistics in every
//                  CTA), and writes its dx segment from shared memory: one
//                  HBM read of each array and one write (Eq. 4, b_reread = 0).
//                  With two row buffers the copies of row r + ncl run while
//                  row r is reduced and written.  The elements past the last
//                  full group (N * size not a multiple of 16) are read from
//                  global memory by the last CTA.
//   k_bwd_tp_*     TWO_PASS: sums over HBM, then a second sweep that rereads
//                  both arrays; G CTAs per row exchange partials through the
//                  device workspace between two launches (G = 1: one fused
//                  kernel, the reread mostly from L2).  Any alignment.
//
// Exchange slots: [parity = row iteration % 2][16 sources][4 floats] ([8
// floats] for the two-input statistics).  A CTA
// pushes its partial for iteration t + 2 into parity t % 2 only after its
// exchange of iteration t + 1 completed, which needed every peer's push of
// t + 1, which each peer made after its own combine of iteration t had read
// those slots; the release fence before each push and the cluster-scope
// acquire of the mbarrier wait carry that order (as in the forward kernels).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_rows.cuh"

namespace credit {
extern std::atomic<long long> g_launch_count;

namespace {

enum BwdOp : int {
    BOP_SOFTMAX = 4, BOP_LN = 5, BOP_RMS = 6, BOP_SMLOGITS = 7, BOP_XENT = 8, BOP_WVAR = 9, BOP_PEARSON = 10
};
template <int OP> constexpr bool kLogits = OP == BOP_SMLOGITS || OP == BOP_XENT;  // online max statistics
template <int OP> constexpr bool kNorm = OP == BOP_LN || OP == BOP_RMS;          // gamma, saved statistics
template <int OP> constexpr bool kPair = OP == BOP_WVAR || OP == BOP_PEARSON;    // two outputs, shifted sums
template <int OP> constexpr int kKind = kLogits<OP> ? 1 : (kPair<OP> ? 2 : 0);
template <int OP> constexpr int kPairState = OP == BOP_WVAR ? 3 : 6;              // centred state of the pair ops

constexpr int kBwdThreads = 512;
constexpr int kBwdCtrl = 1792;             // control area before the row buffers (bytes)
constexpr int kBwdMaxChunks = 8;           // chunks (mbarriers) per row buffer
constexpr uint32_t kBwdPiece = 32768;      // bytes per bulk copy instruction
constexpr long long kBwdFusedMaxBytes = 16384;  // planner: fused two-pass up to this many bytes per array row

struct BwdArgs {
    const unsigned char *a, *dy;
    unsigned char *dx;
    unsigned char *dx2;        // pair ops: the second gradient (dw or dy)
    long long rows, cols, ld;  // ld in elements (all arrays)
    const float *gamma, *mean, *rstd;
    const float *scale;        // cross entropy: per-row upstream scale (null = 1)
    unsigned *err;
    float *ws;                 // two-pass partials [row - row0][G][2] ([G][4] logits ops, [G][8] pair ops)
    int G;                     // two-pass CTAs per row
    int nbuf;                  // staged: row buffers (1 or 2)
    int slice_groups;          // staged: 16-byte groups per array slice buffer
    int gamma_smem;            // staged: this CTA's gamma slice is staged once in shared memory
    int nch, chunk_groups;     // staged: chunks per slice and 16-byte groups per chunk
    long long row0;            // first row of this launch
};

// Per-row constants and the per-element math of each op.
struct Coef {
    float c0, c1, c2, c3, c4;
};

template <int OP>
struct BwdRow {
    float mean = 0.0f, rstd = 1.0f, w = 1.0f;
    __device__ __forceinline__ void load(const BwdArgs &p, long long row) {
        if constexpr (OP == BOP_LN) mean = p.mean[row];
        if constexpr (kNorm<OP>) rstd = p.rstd[row];
        if constexpr (OP == BOP_XENT || kPair<OP>) w = p.scale ? p.scale[row] : 1.0f;
    }
    // pair ops: both gradients of element (a, d)
    __device__ __forceinline__ void dx_pair(float a, float d, const Coef &k, float &o1, float &o2) const {
        if constexpr (OP == BOP_WVAR) {  // c0 = mean, c1 = variance, c2 = g / W
            const float u = a - k.c0;
            o1 = k.c2 * 2.0f * d * u;
            o2 = k.c2 * fmaf(u, u, -k.c1);
        } else {  // c0 = x mean, c1 = y mean, c2 = g / sqrt(Sxx Syy), c3 = g r / Sxx, c4 = g r / Syy
            const float u = a - k.c0, v = d - k.c1;
            o1 = k.c2 * v - k.c3 * u;
            o2 = k.c2 * u - k.c4 * v;
        }
    }
    // add element (a, dy, gamma) to the partial sums
    __device__ __forceinline__ void acc(float a, float d, float gm, float &s0, float &s1) const {
        if constexpr (OP == BOP_SOFTMAX) {
            s0 = fmaf(a, d, s0);
        } else {
            const float g = d * gm;
            const float xh = (OP == BOP_LN ? a - mean : a) * rstd;
            if constexpr (OP == BOP_LN) s0 += g;
            s1 = fmaf(g, xh, s1);
        }
    }
    // dx of element (a, dy, gamma) given the row coefficients: c0 = S0 (softmax) or S0 / N, c1 = S1 / N
    // (norms); c0 = max, c1 = 1 / S, c2 = T / S (softmax from logits); c0 = max, c1 = T / S (cross entropy)
    __device__ __forceinline__ float dx(float a, float d, float gm, const Coef &k) const {
        if constexpr (OP == BOP_SOFTMAX) {
            return a * (d - k.c0);
        } else if constexpr (OP == BOP_SMLOGITS) {
            return exp_fast(a - k.c0) * k.c1 * (d - k.c2);
        } else if constexpr (OP == BOP_XENT) {
            return w * (exp_fast(a - k.c0) * k.c1 - d);
        } else {
            const float g = d * gm;
            const float xh = (OP == BOP_LN ? a - mean : a) * rstd;
            return rstd * (g - k.c0 - xh * k.c1);
        }
    }
};

// Per-thread (and per-CTA) statistics.  Ops 4-6: the plain sums s0, s1.
// Ops 7-8: an online (max m, S = sum exp(z - m), T) triple, T = sum exp(z -
// m) dy (softmax from logits) or sum t (cross entropy); the max of each
// 16-byte group is folded in before its exponentials, as in the forward
// softmax.  merge() is commutative bit for bit, so a shuffle tree gives the
// same state in both lanes of every pair.
template <int OP, int KIND = kKind<OP>>
struct BwdState;

template <int OP>
struct BwdState<OP, 0> {
    float s0 = 0.0f, s1 = 0.0f;
    template <int V>
    __device__ __forceinline__ void add(const BwdRow<OP> &R, const float (&fa)[V], const float (&fd)[V],
                                        const float (&fg)[V]) {
#pragma unroll
        for (int v = 0; v < V; ++v) R.acc(fa[v], fd[v], fg[v], s0, s1);
    }
    __device__ __forceinline__ void add1(const BwdRow<OP> &R, float a, float d, float g) { R.acc(a, d, g, s0, s1); }
};

template <int OP>
struct BwdState<OP, 1> {
    float m = -INFINITY, S = 0.0f, T = 0.0f;
    template <int V>
    __device__ __forceinline__ void add(const BwdRow<OP> &, const float (&fa)[V], const float (&fd)[V],
                                        const float (&)[V]) {
        if constexpr (OP == BOP_XENT) {
#pragma unroll
            for (int v = 0; v < V; ++v) T += fd[v];
        }
        float mv = fa[0];
#pragma unroll
        for (int v = 1; v < V; ++v) mv = fmaxf(mv, fa[v]);
        if (mv == -INFINITY) return;
        if (mv > m) {
            const float r = exp_fast(m - mv);
            S *= r;
            if constexpr (OP == BOP_SMLOGITS) T *= r;
            m = mv;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float e = exp_fast(fa[v] - m);
            S += e;
            if constexpr (OP == BOP_SMLOGITS) T = fmaf(e, fd[v], T);
        }
    }
    __device__ __forceinline__ void add1(const BwdRow<OP> &R, float a, float d, float g) {
        const float fa[1] = {a}, fd[1] = {d}, fg[1] = {g};
        add<1>(R, fa, fd, fg);
    }
    __device__ __forceinline__ void merge(float m2, float S2, float T2) {
        if constexpr (OP == BOP_XENT) T += T2;
        if (S2 == 0.0f) return;
        if (S == 0.0f) {
            m = m2;
            S = S2;
            if constexpr (OP == BOP_SMLOGITS) T = T2;
            return;
        }
        const float M = fmaxf(m, m2), ra = exp_fast(m - M), rb = exp_fast(m2 - M);
        S = S * ra + S2 * rb;
        if constexpr (OP == BOP_SMLOGITS) T = T * ra + T2 * rb;
        m = M;
    }
};

// Pair ops, centred state c[] (weighted variance: W = sum w, mu, M2 = sum w
// (x - mu)^2; Pearson: n, xb, yb and the centred co-moments Sxx, Syy, Sxy).
// c[0] == 0 is the empty state.  Chan's merge of b into a: with n = na + nb
// and the mean differences d = mean_b - mean_a,
//   mean += d nb / n,   S += S_b + d d' na nb / n
// (d' = d of the other variable for the cross moment).  merge(a, b) is the
// same arithmetic whichever side calls it, so the shuffle trees below give
// one state in every lane.  The two weights share one SFU reciprocal of n
// (relative error below 2^-22, as in the LayerNorm statistics).
template <int OP>
__device__ __forceinline__ void pair_merge(float (&a)[kPairState<OP>], const float (&b)[kPairState<OP>]) {
    constexpr int NS = kPairState<OP>;
    if (b[0] == 0.0f) return;
    if (a[0] == 0.0f) {
#pragma unroll
        for (int j = 0; j < NS; ++j) a[j] = b[j];
        return;
    }
    const float n = a[0] + b[0];
    const float wb = b[0] * rcp_approx(n), wab = a[0] * wb;  // nb / n and na nb / n
    if constexpr (OP == BOP_WVAR) {
        const float d = b[1] - a[1];
        a[1] = fmaf(d, wb, a[1]);
        a[2] = a[2] + b[2] + d * d * wab;
    } else {
        const float dx = b[1] - a[1], dy = b[2] - a[2];
        a[1] = fmaf(dx, wb, a[1]);
        a[2] = fmaf(dy, wb, a[2]);
        a[3] = a[3] + b[3] + dx * dx * wab;
        a[4] = a[4] + b[4] + dy * dy * wab;
        a[5] = a[5] + b[5] + dx * dy * wab;
    }
    a[0] = n;
}

// Pair ops, per thread: sums about the thread's first element of each array
// (kx, ky), so the second moments lose little to cancellation, converted once
// by finish() to the centred state (the scheme of the forward LayerNorm
// statistics).  Weighted variance: W, sum w u, sum w u^2 (u = x - kx);
// Pearson: n, sum u, sum v, sum u^2, sum v^2, sum u v (v = y - ky).
template <int OP>
struct BwdState<OP, 2> {
    float n = 0.0f, kx = 0.0f, ky = 0.0f;
    float s[5] = {};
    bool has = false;
    __device__ __forceinline__ void acc(float a, float d) {
        if (!has) {
            kx = a;
            ky = d;
            has = true;
        }
        if constexpr (OP == BOP_WVAR) {  // d is the weight
            const float u = a - kx, wu = d * u;
            n += d;
            s[0] += wu;
            s[1] = fmaf(wu, u, s[1]);
        } else {
            const float u = a - kx, v = d - ky;
            n += 1.0f;
            s[0] += u;
            s[1] += v;
            s[2] = fmaf(u, u, s[2]);
            s[3] = fmaf(v, v, s[3]);
            s[4] = fmaf(u, v, s[4]);
        }
    }
    template <int V>
    __device__ __forceinline__ void add(const BwdRow<OP> &, const float (&fa)[V], const float (&fd)[V],
                                        const float (&)[V]) {
#pragma unroll
        for (int v = 0; v < V; ++v) acc(fa[v], fd[v]);
    }
    __device__ __forceinline__ void add1(const BwdRow<OP> &, float a, float d, float) { acc(a, d); }
    __device__ __forceinline__ void finish(float (&c)[kPairState<OP>]) const {
#pragma unroll
        for (int j = 0; j < kPairState<OP>; ++j) c[j] = 0.0f;
        if (n == 0.0f) return;
        const float r = rcp_approx(n);
        if constexpr (OP == BOP_WVAR) {
            const float q = s[0] * r;
            c[0] = n;
            c[1] = kx + q;
            c[2] = fmaxf(fmaf(-s[0], q, s[1]), 0.0f);
        } else {
            const float qx = s[0] * r, qy = s[1] * r;
            c[0] = n;
            c[1] = kx + qx;
            c[2] = ky + qy;
            c[3] = fmaxf(fmaf(-s[0], qx, s[2]), 0.0f);
            c[4] = fmaxf(fmaf(-s[1], qy, s[3]), 0.0f);
            c[5] = fmaf(-s[0], qy, s[4]);
        }
    }
};

// Shuffle-tree merge of a pair state over groups of `width` lanes (a power
// of two, <= 32): at every level both partners compute merge(lower lane,
// upper lane), so all lanes of a group end with the same state.
template <int OP>
__device__ __forceinline__ void warp_merge_pair(float (&c)[kPairState<OP>], int width = 32) {
    constexpr int NS = kPairState<OP>;
    const int lane = threadIdx.x & 31;
    for (int o = width >> 1; o > 0; o >>= 1) {
        float oth[NS];
#pragma unroll
        for (int j = 0; j < NS; ++j) oth[j] = __shfl_xor_sync(0xffffffffu, c[j], o);
        if (lane & o) {
            pair_merge<OP>(oth, c);
#pragma unroll
            for (int j = 0; j < NS; ++j) c[j] = oth[j];
        } else {
            pair_merge<OP>(c, oth);
        }
    }
}

// Deterministic block merge of the threads' pair states through red (>= 17 NS
// floats): a shuffle tree per warp, then one over the warps' states in warp 0.
// Every thread returns the CTA's state in out.  Contains two __syncthreads.
template <int OP>
__device__ __forceinline__ void block_merge_pair(const BwdState<OP, 2> &st, float *red,
                                                 float (&out)[kPairState<OP>]) {
    constexpr int NS = kPairState<OP>;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float c[NS];
    st.finish(c);
    warp_merge_pair<OP>(c);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NS; ++j) red[NS * wid + j] = c[j];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int j = 0; j < NS; ++j) c[j] = lane < nw ? red[NS * lane + j] : 0.0f;
        warp_merge_pair<OP>(c);
        if (lane == 0) {
#pragma unroll
            for (int j = 0; j < NS; ++j) red[NS * 16 + j] = c[j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NS; ++j) out[j] = red[NS * 16 + j];
}

// Coefficients of the pair ops from the row's centred state (see BwdRow::dx_pair).
template <int OP>
__device__ __forceinline__ Coef pair_coeffs(const float (&t)[kPairState<OP>], const BwdRow<OP> &R) {
    if constexpr (OP == BOP_WVAR) {
        const float inv = 1.0f / t[0];
        return {t[1], t[2] * inv, R.w * inv, 0.0f, 0.0f};
    } else {
        const float inv_den = 1.0f / (sqrtf(t[3]) * sqrtf(t[4])), r = t[5] * inv_den;
        return {t[1], t[2], R.w * inv_den, R.w * r / t[3], R.w * r / t[4]};
    }
}

// Push all-gather of up to 8 floats per CTA: slots of 8 floats, [par][16][8],
// two 16-byte st.async per peer (the protocol of exchange_push).
__device__ __forceinline__ const float *exchange_push8(const float (&v)[8], float *slots, uint64_t *xbar, int par,
                                                       uint32_t phase, int P, int c, int Tc, unsigned *err) {
    const int tid = threadIdx.x;
    float *base = slots + par * 16 * 8;
    float *mine = base + c * 8;
    uint64_t *bar = &xbar[par];
    if (tid < P) {
        if (tid == c) {
#pragma unroll
            for (int j = 0; j < 8; ++j) mine[j] = v[j];
        } else {
            fence_release_smem_cluster();
            const uint32_t raddr = mapa_shared(smem_addr(mine), static_cast<uint32_t>(tid));
            const uint32_t rbar = mapa_shared(smem_addr(bar), static_cast<uint32_t>(tid));
            st_async_v4f32(raddr, make_float4(v[0], v[1], v[2], v[3]), rbar);
            st_async_v4f32(raddr + 16, make_float4(v[4], v[5], v[6], v[7]), rbar);
        }
    }
    if (tid == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>((P - 1) * 32));
    named_bar_sync(1, Tc);
    mbar_wait_bounded_cluster(bar, phase, err);
    return base;
}

template <int OP>
__device__ __forceinline__ Coef logit_coeffs(float M, float S, float T) {
    const float inv = 1.0f / S;
    if constexpr (OP == BOP_SMLOGITS) return {M, inv, T * inv, 0.0f, 0.0f};
    else return {M, T * inv, 0.0f, 0.0f, 0.0f};
}

// Shuffle-tree merge of the logits state over groups of `width` lanes (a
// power of two).  The tree is fixed and merge() commutative, so every lane
// of a group ends with the same state; merging an empty state is exact.
template <int OP>
__device__ __forceinline__ void warp_merge_logits(BwdState<OP, 1> &st, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) {
        const float m2 = __shfl_xor_sync(0xffffffffu, st.m, o);
        const float S2 = __shfl_xor_sync(0xffffffffu, st.S, o);
        const float T2 = __shfl_xor_sync(0xffffffffu, st.T, o);
        st.merge(m2, S2, T2);
    }
}

// Deterministic block merge of the logits state through red (>= 67 floats):
// a shuffle tree per warp, then one over the warps' states in warp 0.  Every
// thread returns (m, S, T, 0).  Contains two __syncthreads.
template <int OP>
__device__ __forceinline__ float4 block_reduce_logits(BwdState<OP, 1> st, float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    warp_merge_logits<OP>(st, 32);
    if (lane == 0) {
        red[4 * wid] = st.m;
        red[4 * wid + 1] = st.S;
        red[4 * wid + 2] = st.T;
    }
    __syncthreads();
    if (wid == 0) {
        BwdState<OP, 1> t;
        if (lane < nw) {
            t.m = red[4 * lane];
            t.S = red[4 * lane + 1];
            t.T = red[4 * lane + 2];
        }
        warp_merge_logits<OP>(t, 32);
        if (lane == 0) {
            red[64] = t.m;
            red[65] = t.S;
            red[66] = t.T;
        }
    }
    __syncthreads();
    return make_float4(red[64], red[65], red[66], 0.0f);
}

// Push all-gather of one 16-byte partial per CTA (the logits ops' triple),
// the same protocol as exchange_push: own slot written locally, peers' slots
// by st.async completing on their exchange mbarrier, after a release fence
// that orders this CTA's earlier reads of its slots.
__device__ __forceinline__ const float *exchange_push4(const float4 &v, float *slots, uint64_t *xbar, int par,
                                                       uint32_t phase, int P, int c, int Tc, unsigned *err) {
    const int tid = threadIdx.x;
    float *mine = slot_ptr(slots, 0, par, c);
    uint64_t *bar = &xbar[par];
    if (tid < P) {
        if (tid == c) {
            mine[0] = v.x;
            mine[1] = v.y;
            mine[2] = v.z;
            mine[3] = v.w;
        } else {
            fence_release_smem_cluster();
            const uint32_t raddr = mapa_shared(smem_addr(mine), static_cast<uint32_t>(tid));
            const uint32_t rbar = mapa_shared(smem_addr(bar), static_cast<uint32_t>(tid));
            st_async_v4f32(raddr, v, rbar);
        }
    }
    if (tid == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>((P - 1) * 16));
    named_bar_sync(1, Tc);
    mbar_wait_bounded_cluster(bar, phase, err);
    return slot_ptr(slots, 0, par, 0);
}

// Coefficients of ops 4-6 from the row totals (S0, S1) and N.
template <int OP>
__device__ __forceinline__ Coef row_coeffs(float S0, float S1, long long N) {
    const float inv_n = 1.0f / static_cast<float>(N);
    if constexpr (OP == BOP_SOFTMAX) return {S0, 0.0f, 0.0f, 0.0f, 0.0f};
    else if constexpr (OP == BOP_LN) return {S0 * inv_n, S1 * inv_n, 0.0f, 0.0f, 0.0f};
    else return {0.0f, S1 * inv_n, 0.0f, 0.0f, 0.0f};
}

// Deterministic block sum of two floats through red (>= 66 floats); every
// thread returns the totals.  Contains two __syncthreads.
__device__ __forceinline__ float2 block_sum2(float a, float b, float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane == 0) {
        red[2 * wid] = a;
        red[2 * wid + 1] = b;
    }
    __syncthreads();
    if (wid == 0) {
        float ta = lane < nw ? red[2 * lane] : 0.0f;
        float tb = lane < nw ? red[2 * lane + 1] : 0.0f;
        ta = warp_sum(ta);
        tb = warp_sum(tb);
        if (lane == 0) {
            red[64] = ta;
            red[65] = tb;
        }
    }
    __syncthreads();
    return make_float2(red[64], red[65]);
}

// ------------------------------------------------------------------ staged (ONE_CTA / CLUSTER)
// Shared memory: [0, 128) full[2][8] mbarriers (row buffer x chunk), [128,
// 144) xbar[2] mbarriers, [144, 152) gbar mbarrier, [256, 768) reduction
// scratch, [768, 1280) exchange slots, then nbuf row buffers of (a slice, dy
// slice), slice_groups * 16 bytes each, then (gamma_smem) the CTA's FP32
// gamma slice, staged once for all rows: gamma is the same for every row, so
// the loops read it from shared memory instead of issuing an L2 load per
// element group.
//
// A slice is processed in nch chunks of chunk_groups groups, each with its
// own mbarrier, so the sweep starts on chunk 0 while later chunks land.  With
// two row buffers the whole next row is issued into the other buffer when a
// row starts.  With one buffer (slices too large for two) chunk q of the next
// row is issued as soon as every thread has written its outputs of chunk q of
// this row, so the copies of the next row overlap this row's write pass.
template <int OP, int DT>
__global__ void __launch_bounds__(kBwdThreads, 1) k_bwd_staged(const BwdArgs p) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);  // [b * kBwdMaxChunks + q]
    uint64_t *xbar = full + 2 * kBwdMaxChunks;
    uint64_t *gbar = xbar + 2;
    float *red = reinterpret_cast<float *>(smem + 256);
    float *slots = reinterpret_cast<float *>(smem + 768);
    unsigned char *data = smem + kBwdCtrl;
    constexpr int isz = Fmt<DT>::size, V = Fmt<DT>::V;
    constexpr int NQ = (OP == BOP_LN) ? 2 : 1;

    const int P = static_cast<int>(cluster_nctarank());
    const int c = static_cast<int>(cluster_ctarank());
    const long long cl = blockIdx.x / P, ncl = gridDim.x / P;
    const int tid = threadIdx.x, T = blockDim.x;
    const long long N = p.cols;
    const long long Gq = N / V;                  // full 16-byte groups of a row
    const long long tail = N - Gq * V;
    const long long g_lo = group_split(Gq, c, P), g_hi = group_split(Gq, c + 1, P);
    const int ng = static_cast<int>(g_hi - g_lo);
    const int nch = p.nch, cg = p.chunk_groups;
    const size_t arr = static_cast<size_t>(p.slice_groups) * 16;
    const bool g_vec = p.gamma == nullptr || (reinterpret_cast<uintptr_t>(p.gamma) & 15u) == 0;
    const bool g_sm = kNorm<OP> && p.gamma_smem;
    const float *gs = reinterpret_cast<const float *>(data + static_cast<size_t>(p.nbuf) * 2 * arr);

    if (tid == 0) {
        for (int k = 0; k < 2 * kBwdMaxChunks; ++k) mbar_init(&full[k], 1);
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
        mbar_init(gbar, 1);
        fence_mbar_init();
        if (g_sm) {  // this CTA's gamma slice, once
            const uint32_t gbytes = static_cast<uint32_t>(ng) * V * 4u;
            mbar_arrive_expect_tx(gbar, gbytes);
            for (uint32_t o = 0; o < gbytes; o += kBwdPiece) {
                const uint32_t n = gbytes - o < kBwdPiece ? gbytes - o : kBwdPiece;
                bulk_g2s(reinterpret_cast<unsigned char *>(const_cast<float *>(gs)) + o,
                         reinterpret_cast<const unsigned char *>(p.gamma + g_lo * V) + o, n, gbar);
            }
        }
    }
    __syncthreads();
    if (g_sm) mbar_wait_bounded(gbar, 0, p.err);
    if (P > 1) {  // every peer's exchange barriers exist before the first push
        cluster_arrive_release();
        cluster_wait_acquire();
    }

    // groups [k0, k1) of chunk q of this CTA's slice
    auto chunk_range = [&](int q, int &k0, int &k1) {
        k0 = q * cg < ng ? q * cg : ng;
        k1 = (q + 1) * cg < ng ? (q + 1) * cg : ng;
    };
    // thread 0: stage chunk q of this CTA's slices of row `row` into buffer b
    auto issue_chunk = [&](long long row, int b, int q) {
        int k0, k1;
        chunk_range(q, k0, k1);
        const size_t off = static_cast<size_t>(row * p.ld + (g_lo + k0) * V) * isz;
        unsigned char *da = data + static_cast<size_t>(b) * 2 * arr + static_cast<size_t>(k0) * 16;
        unsigned char *dd = da + arr;
        const uint32_t bytes = static_cast<uint32_t>(k1 - k0) * 16u;
        uint64_t *bar = &full[b * kBwdMaxChunks + q];
        mbar_arrive_expect_tx(bar, 2 * bytes);
        for (uint32_t o = 0; o < bytes; o += kBwdPiece) {
            const uint32_t n = bytes - o < kBwdPiece ? bytes - o : kBwdPiece;
            bulk_g2s(da + o, p.a + off + o, n, bar);
            bulk_g2s(dd + o, p.dy + off + o, n, bar);
        }
    };

    if (tid == 0 && cl < p.rows)
        for (int q = 0; q < nch; ++q) issue_chunk(cl, 0, q);
    long long it = 0;
    for (long long row = cl; row < p.rows; row += ncl, ++it) {
        const int b = p.nbuf == 2 ? static_cast<int>(it & 1) : 0;
        const uint32_t fpar = p.nbuf == 2 ? static_cast<uint32_t>((it >> 1) & 1) : static_cast<uint32_t>(it & 1);
        const bool more = row + ncl < p.rows;
        // two buffers: the whole next row into the other one (read last in the previous iteration, before
        // that iteration's final barrier)
        if (p.nbuf == 2 && tid == 0 && more) {
            fence_proxy_async_smem();
            for (int q = 0; q < nch; ++q) issue_chunk(row + ncl, b ^ 1, q);
        }
        BwdRow<OP> R;
        R.load(p, row);
        const unsigned char *da = data + static_cast<size_t>(b) * 2 * arr, *dd = da + arr;
        const size_t row_off = static_cast<size_t>(row * p.ld) * isz;

        BwdState<OP> st;
        auto sweep = [&](int k0, int k1) {
            for (int k = k0 + tid; k < k1; k += T) {
                float fa[V], fd[V], fg[V];
                decode_group<DT>(*reinterpret_cast<const uint4 *>(da + 16 * k), fa, 1.0f);
                decode_group<DT>(*reinterpret_cast<const uint4 *>(dd + 16 * k), fd, 1.0f);
                if (g_sm) load_affine_smem<V>(gs, k * V, 1.0f, fg);
                else load_affine<V>(kNorm<OP> ? p.gamma : nullptr, (g_lo + k) * V, g_vec, 1.0f, fg);
                st.template add<V>(R, fa, fd, fg);
            }
        };
        if (nch == 1) {
            mbar_wait_bounded(&full[b * kBwdMaxChunks], fpar, p.err);
            sweep(0, ng);
        } else {
            for (int q = 0; q < nch; ++q) {
                int k0, k1;
                chunk_range(q, k0, k1);
                mbar_wait_bounded(&full[b * kBwdMaxChunks + q], fpar, p.err);
                sweep(k0, k1);
            }
        }
        if (c == P - 1) {
            for (long long t = tid; t < tail; t += T) {
                const long long i = Gq * V + t;
                const float gm = (kNorm<OP> && p.gamma) ? p.gamma[i] : 1.0f;
                st.add1(R, decode_one<DT>(p.a + row_off + i * isz, 1.0f),
                        decode_one<DT>(p.dy + row_off + i * isz, 1.0f), gm);
            }
        }
        Coef kc;
        if constexpr (kPair<OP>) {
            constexpr int NS = kPairState<OP>;
            float tot[NS];
            block_merge_pair<OP>(st, red, tot);
            if (P > 1) {
                float v8[8] = {};
#pragma unroll
                for (int j = 0; j < NS; ++j) v8[j] = tot[j];
                const float *sl = exchange_push8(v8, slots, xbar, static_cast<int>(it & 1),
                                                 static_cast<uint32_t>((it >> 1) & 1), P, c, T, p.err);
                // the P CTA states merged by one fixed shuffle tree within every group of P lanes (lane l
                // holds CTA l % P's; P is a power of two): the same state in every thread of every CTA
                const int q = tid & (P - 1);
#pragma unroll
                for (int j = 0; j < NS; ++j) tot[j] = sl[8 * q + j];
                warp_merge_pair<OP>(tot, P);
            }
            kc = pair_coeffs<OP>(tot, R);
        } else if constexpr (kLogits<OP>) {
            float4 tot = block_reduce_logits<OP>(st, red);
            if (P > 1) {
                const float *sl = exchange_push4(tot, slots, xbar, static_cast<int>(it & 1),
                                                 static_cast<uint32_t>((it >> 1) & 1), P, c, T, p.err);
                // the P partials merged by one fixed shuffle tree (lane q holds CTA q's): the same state in
                // every thread of every CTA of the cluster
                BwdState<OP> all;
                const int lane = tid & 31;
                if (lane < P) {
                    all.m = sl[4 * lane];
                    all.S = sl[4 * lane + 1];
                    all.T = sl[4 * lane + 2];
                }
                warp_merge_logits<OP>(all, 32);  // merging an empty state changes nothing
                tot = make_float4(all.m, all.S, all.T, 0.0f);
            }
            kc = logit_coeffs<OP>(tot.x, tot.y, tot.z);
        } else {
            float2 tot = block_sum2(st.s0, st.s1, red);
            if (P > 1) {
                const float *sl = exchange_push<NQ>(OP == BOP_RMS ? tot.y : tot.x, tot.y, slots, xbar, 0,
                                                    static_cast<int>(it & 1), static_cast<uint32_t>((it >> 1) & 1),
                                                    P, c, T, p.err);
                float S0 = 0.0f, S1 = 0.0f;
                for (int q = 0; q < P; ++q) {  // fixed order: the same totals in every CTA
                    S0 += sl[4 * q];
                    if (NQ == 2) S1 += sl[4 * q + 1];
                }
                tot = OP == BOP_RMS ? make_float2(0.0f, S0) : make_float2(S0, S1);
            }
            kc = row_coeffs<OP>(tot.x, tot.y, N);
        }
        if (c == P - 1) {  // the elements past the last full group, from global memory
            for (long long t = tid; t < tail; t += T) {
                const long long i = Gq * V + t;
                const float gm = (kNorm<OP> && p.gamma) ? p.gamma[i] : 1.0f;
                const float av = decode_one<DT>(p.a + row_off + i * isz, 1.0f);
                const float dv = decode_one<DT>(p.dy + row_off + i * isz, 1.0f);
                if constexpr (kPair<OP>) {
                    float o1, o2;
                    R.dx_pair(av, dv, kc, o1, o2);
                    store_one<DT>(p.dx + row_off + i * isz, o1);
                    store_one<DT>(p.dx2 + row_off + i * isz, o2);
                } else {
                    store_one<DT>(p.dx + row_off + i * isz, R.dx(av, dv, gm, kc));
                }
            }
        }
        unsigned char *xr = p.dx + row_off + static_cast<size_t>(g_lo * V) * isz;
        unsigned char *xr2 = kPair<OP> ? p.dx2 + row_off + static_cast<size_t>(g_lo * V) * isz : nullptr;
        auto write = [&](int k0, int k1) {
            for (int k = k0 + tid; k < k1; k += T) {
                float fa[V], fd[V], fg[V], y[V];
                decode_group<DT>(*reinterpret_cast<const uint4 *>(da + 16 * k), fa, 1.0f);
                decode_group<DT>(*reinterpret_cast<const uint4 *>(dd + 16 * k), fd, 1.0f);
                if (g_sm) load_affine_smem<V>(gs, k * V, 1.0f, fg);
                else load_affine<V>(kNorm<OP> ? p.gamma : nullptr, (g_lo + k) * V, g_vec, 1.0f, fg);
                if constexpr (kPair<OP>) {
                    float y2[V];
#pragma unroll
                    for (int v = 0; v < V; ++v) R.dx_pair(fa[v], fd[v], kc, y[v], y2[v]);
                    store_group<DT, V>(xr + 16 * k, y, true);
                    store_group<DT, V>(xr2 + 16 * k, y2, true);
                } else {
#pragma unroll
                    for (int v = 0; v < V; ++v) y[v] = R.dx(fa[v], fd[v], fg[v], kc);
                    store_group<DT, V>(xr + 16 * k, y, true);
                }
            }
        };
        if (p.nbuf == 2) {
            write(0, ng);
            __syncthreads();  // every read of buffer b is done before it is refilled
        } else {
            for (int q = 0; q < nch; ++q) {
                int k0, k1;
                chunk_range(q, k0, k1);
                write(k0, k1);
                __syncthreads();  // every read of chunk q is done before it is refilled
                if (tid == 0 && more) {
                    fence_proxy_async_smem();
                    issue_chunk(row + ncl, 0, q);
                }
            }
        }
    }
    if (P > 1) {  // nobody exits while a peer may still push into it
        cluster_arrive_release();
        cluster_wait_acquire();
    }
}

// ------------------------------------------------------------------ two-pass
// Units of CTA j of G for one row: 16-byte groups when the row's three
// arrays are 16-byte aligned (plus the tail elements, by CTA G - 1), single
// elements otherwise.
struct BwdSpan {
    bool vec;
    long long lo, hi;        // groups (vec) or elements
    long long t_lo, t_hi;    // tail elements handled here (vec only)
};

template <int DT>
__device__ __forceinline__ BwdSpan bwd_span(const BwdArgs &p, long long row, int j, int G) {
    constexpr int isz = Fmt<DT>::size, V = Fmt<DT>::V;
    const size_t off = static_cast<size_t>(row * p.ld) * isz;
    const bool vec = ((reinterpret_cast<uintptr_t>(p.a + off) | reinterpret_cast<uintptr_t>(p.dy + off) |
                       reinterpret_cast<uintptr_t>(p.dx + off) |
                       (p.dx2 ? reinterpret_cast<uintptr_t>(p.dx2 + off) : 0)) & 15u) == 0;
    BwdSpan s;
    s.vec = vec;
    if (vec) {
        const long long Gq = p.cols / V;
        s.lo = group_split(Gq, j, G);
        s.hi = group_split(Gq, j + 1, G);
        s.t_lo = j == G - 1 ? Gq * V : p.cols;
        s.t_hi = p.cols;
    } else {
        s.lo = group_split(p.cols, j, G);
        s.hi = group_split(p.cols, j + 1, G);
        s.t_lo = s.t_hi = 0;
    }
    return s;
}

template <int OP, int DT>
__device__ __forceinline__ BwdState<OP> bwd_sums(const BwdArgs &p, long long row, const BwdRow<OP> &R,
                                                 const BwdSpan &s) {
    constexpr int isz = Fmt<DT>::size, V = Fmt<DT>::V;
    const size_t off = static_cast<size_t>(row * p.ld) * isz;
    const bool g_vec = p.gamma == nullptr || (reinterpret_cast<uintptr_t>(p.gamma) & 15u) == 0;
    const float *gam = kNorm<OP> ? p.gamma : nullptr;
    BwdState<OP> st;
    if (s.vec) {
        for (long long k = s.lo + threadIdx.x; k < s.hi; k += blockDim.x) {
            float fa[V], fd[V], fg[V];
            decode_group<DT>(ld_global_v4(p.a + off + 16 * k), fa, 1.0f);
            decode_group<DT>(ld_global_v4(p.dy + off + 16 * k), fd, 1.0f);
            load_affine<V>(gam, k * V, g_vec, 1.0f, fg);
            st.template add<V>(R, fa, fd, fg);
        }
    }
    const long long e_lo = s.vec ? s.t_lo : s.lo, e_hi = s.vec ? s.t_hi : s.hi;
    for (long long i = e_lo + threadIdx.x; i < e_hi; i += blockDim.x)
        st.add1(R, decode_one<DT>(p.a + off + i * isz, 1.0f), decode_one<DT>(p.dy + off + i * isz, 1.0f),
                gam ? gam[i] : 1.0f);
    return st;
}

template <int OP, int DT>
__device__ __forceinline__ void bwd_apply(const BwdArgs &p, long long row, const BwdRow<OP> &R, const BwdSpan &s,
                                          const Coef &kc) {
    constexpr int isz = Fmt<DT>::size, V = Fmt<DT>::V;
    const size_t off = static_cast<size_t>(row * p.ld) * isz;
    const bool g_vec = p.gamma == nullptr || (reinterpret_cast<uintptr_t>(p.gamma) & 15u) == 0;
    const float *gam = kNorm<OP> ? p.gamma : nullptr;
    if (s.vec) {
        for (long long k = s.lo + threadIdx.x; k < s.hi; k += blockDim.x) {
            float fa[V], fd[V], fg[V], y[V];
            decode_group<DT>(ld_global_v4(p.a + off + 16 * k), fa, 1.0f);
            decode_group<DT>(ld_global_v4(p.dy + off + 16 * k), fd, 1.0f);
            load_affine<V>(gam, k * V, g_vec, 1.0f, fg);
            if constexpr (kPair<OP>) {
                float y2[V];
#pragma unroll
                for (int v = 0; v < V; ++v) R.dx_pair(fa[v], fd[v], kc, y[v], y2[v]);
                store_group<DT, V>(p.dx + off + 16 * k, y, true);
                store_group<DT, V>(p.dx2 + off + 16 * k, y2, true);
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) y[v] = R.dx(fa[v], fd[v], fg[v], kc);
                store_group<DT, V>(p.dx + off + 16 * k, y, true);
            }
        }
    }
    const long long e_lo = s.vec ? s.t_lo : s.lo, e_hi = s.vec ? s.t_hi : s.hi;
    for (long long i = e_lo + threadIdx.x; i < e_hi; i += blockDim.x) {
        const float av = decode_one<DT>(p.a + off + i * isz, 1.0f), dv = decode_one<DT>(p.dy + off + i * isz, 1.0f);
        if constexpr (kPair<OP>) {
            float o1, o2;
            R.dx_pair(av, dv, kc, o1, o2);
            store_one<DT>(p.dx + off + i * isz, o1);
            store_one<DT>(p.dx2 + off + i * isz, o2);
        } else {
            store_one<DT>(p.dx + off + i * isz, R.dx(av, dv, gam ? gam[i] : 1.0f, kc));
        }
    }
}

// G = 1: one CTA per row, both sweeps.
template <int OP, int DT>
__global__ void __launch_bounds__(kBwdThreads) k_bwd_tp_fused(const BwdArgs p) {
    __shared__ float red[128];
    const long long row = p.row0 + blockIdx.x;
    BwdRow<OP> R;
    R.load(p, row);
    const BwdSpan s = bwd_span<DT>(p, row, 0, 1);
    const BwdState<OP> t = bwd_sums<OP, DT>(p, row, R, s);
    Coef kc;
    if constexpr (kPair<OP>) {
        float tot[kPairState<OP>];
        block_merge_pair<OP>(t, red, tot);
        kc = pair_coeffs<OP>(tot, R);
    } else if constexpr (kLogits<OP>) {
        const float4 tot = block_reduce_logits<OP>(t, red);
        kc = logit_coeffs<OP>(tot.x, tot.y, tot.z);
    } else {
        const float2 tot = block_sum2(t.s0, t.s1, red);
        kc = row_coeffs<OP>(tot.x, tot.y, p.cols);
    }
    bwd_apply<OP, DT>(p, row, R, s, kc);
}

// G > 1, launch 1: partial sums of CTA j of row lr into ws[lr][j][0..1] (logits ops: the state into
// ws[lr][j][0..2] of a 4-float record; pair ops: the sums into an 8-float record).
template <int OP, int DT>
__global__ void __launch_bounds__(kBwdThreads) k_bwd_tp_stats(const BwdArgs p) {
    __shared__ float red[128];
    const int G = p.G, j = blockIdx.x % G;
    const long long lr = blockIdx.x / G, row = p.row0 + lr;
    BwdRow<OP> R;
    R.load(p, row);
    const BwdSpan s = bwd_span<DT>(p, row, j, G);
    const BwdState<OP> t = bwd_sums<OP, DT>(p, row, R, s);
    if constexpr (kPair<OP>) {
        float tot[kPairState<OP>];
        block_merge_pair<OP>(t, red, tot);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < kPairState<OP>; ++q) p.ws[(lr * G + j) * 8 + q] = tot[q];
        }
    } else if constexpr (kLogits<OP>) {
        const float4 tot = block_reduce_logits<OP>(t, red);
        if (threadIdx.x == 0) {
            p.ws[(lr * G + j) * 4] = tot.x;
            p.ws[(lr * G + j) * 4 + 1] = tot.y;
            p.ws[(lr * G + j) * 4 + 2] = tot.z;
        }
    } else {
        const float2 tot = block_sum2(t.s0, t.s1, red);
        if (threadIdx.x == 0) {
            p.ws[(lr * G + j) * 2] = tot.x;
            p.ws[(lr * G + j) * 2 + 1] = tot.y;
        }
    }
}

// G > 1, launch 2: the row totals (partials in the fixed order j = 0..G-1), then dx.
template <int OP, int DT>
__global__ void __launch_bounds__(kBwdThreads) k_bwd_tp_apply(const BwdArgs p) {
    const int G = p.G, j = blockIdx.x % G;
    const long long lr = blockIdx.x / G, row = p.row0 + lr;
    BwdRow<OP> R;
    R.load(p, row);
    Coef kc;
    if constexpr (kPair<OP>) {
        float tot[kPairState<OP>] = {};
        for (int q = 0; q < G; ++q) {  // Chan merges in the fixed order j = 0..G-1
            float cq[kPairState<OP>];
#pragma unroll
            for (int i = 0; i < kPairState<OP>; ++i) cq[i] = p.ws[(lr * G + q) * 8 + i];
            pair_merge<OP>(tot, cq);
        }
        kc = pair_coeffs<OP>(tot, R);
    } else if constexpr (kLogits<OP>) {
        BwdState<OP> all;
        for (int q = 0; q < G; ++q)
            all.merge(p.ws[(lr * G + q) * 4], p.ws[(lr * G + q) * 4 + 1], p.ws[(lr * G + q) * 4 + 2]);
        kc = logit_coeffs<OP>(all.m, all.S, all.T);
    } else {
        float S0 = 0.0f, S1 = 0.0f;
        for (int q = 0; q < G; ++q) {
            S0 += p.ws[(lr * G + q) * 2];
            S1 += p.ws[(lr * G + q) * 2 + 1];
        }
        kc = row_coeffs<OP>(S0, S1, p.cols);
    }
    bwd_apply<OP, DT>(p, row, R, bwd_span<DT>(p, row, j, G), kc);
}

struct BwdKernels {
    const void *staged, *fused, *stats, *apply;
};

template <int OP, int DT>
BwdKernels bwd_kernels_of() {
    return {reinterpret_cast<const void *>(&k_bwd_staged<OP, DT>), reinterpret_cast<const void *>(&k_bwd_tp_fused<OP, DT>),
            reinterpret_cast<const void *>(&k_bwd_tp_stats<OP, DT>),
            reinterpret_cast<const void *>(&k_bwd_tp_apply<OP, DT>)};
}

bool bwd_kernels(int op, int dt, BwdKernels *k) {
    switch (op * 4 + dt) {
    case BOP_SOFTMAX * 4 + DT_F32: *k = bwd_kernels_of<BOP_SOFTMAX, DT_F32>(); return true;
    case BOP_SOFTMAX * 4 + DT_BF16: *k = bwd_kernels_of<BOP_SOFTMAX, DT_BF16>(); return true;
    case BOP_LN * 4 + DT_F32: *k = bwd_kernels_of<BOP_LN, DT_F32>(); return true;
    case BOP_LN * 4 + DT_BF16: *k = bwd_kernels_of<BOP_LN, DT_BF16>(); return true;
    case BOP_RMS * 4 + DT_F32: *k = bwd_kernels_of<BOP_RMS, DT_F32>(); return true;
    case BOP_RMS * 4 + DT_BF16: *k = bwd_kernels_of<BOP_RMS, DT_BF16>(); return true;
    case BOP_SMLOGITS * 4 + DT_F32: *k = bwd_kernels_of<BOP_SMLOGITS, DT_F32>(); return true;
    case BOP_SMLOGITS * 4 + DT_BF16: *k = bwd_kernels_of<BOP_SMLOGITS, DT_BF16>(); return true;
    case BOP_XENT * 4 + DT_F32: *k = bwd_kernels_of<BOP_XENT, DT_F32>(); return true;
    case BOP_XENT * 4 + DT_BF16: *k = bwd_kernels_of<BOP_XENT, DT_BF16>(); return true;
    case BOP_WVAR * 4 + DT_F32: *k = bwd_kernels_of<BOP_WVAR, DT_F32>(); return true;
    case BOP_WVAR * 4 + DT_BF16: *k = bwd_kernels_of<BOP_WVAR, DT_BF16>(); return true;
    case BOP_PEARSON * 4 + DT_F32: *k = bwd_kernels_of<BOP_PEARSON, DT_F32>(); return true;
    case BOP_PEARSON * 4 + DT_BF16: *k = bwd_kernels_of<BOP_PEARSON, DT_BF16>(); return true;
    default: return false;
    }
}

// ------------------------------------------------------------------ host
credit_status validate_bwd(const credit_bwd_args *a) {
    if (a == nullptr) return CREDIT_ERR_INVALID_ARG;
    if (a->op < BOP_SOFTMAX || a->op > BOP_PEARSON) return CREDIT_ERR_INVALID_ARG;
    if (a->dtype == CREDIT_FP8_E4M3) return CREDIT_ERR_UNSUPPORTED;
    if (a->dtype != CREDIT_F32 && a->dtype != CREDIT_BF16) return CREDIT_ERR_INVALID_ARG;
    if (a->rows < 0 || a->cols <= 0 || a->ld < 0 || (a->ld != 0 && a->ld < a->cols)) return CREDIT_ERR_INVALID_ARG;
    if (a->rows == 0) return CREDIT_OK;
    if (a->a == nullptr || a->dy == nullptr || a->dx == nullptr) return CREDIT_ERR_INVALID_ARG;
    if (a->op == BOP_LN && (a->mean == nullptr || a->rstd == nullptr)) return CREDIT_ERR_INVALID_ARG;
    if (a->op == BOP_RMS && a->rstd == nullptr) return CREDIT_ERR_INVALID_ARG;
    if ((a->op == BOP_WVAR || a->op == BOP_PEARSON) && a->dx2 == nullptr) return CREDIT_ERR_INVALID_ARG;
    return CREDIT_OK;
}

bool rows_aligned(const credit_bwd_args *a) {
    const long long ld = a->ld ? a->ld : a->cols;
    const int isz = dtype_size(a->dtype);
    const uintptr_t u = reinterpret_cast<uintptr_t>(a->a) | reinterpret_cast<uintptr_t>(a->dy) |
                        reinterpret_cast<uintptr_t>(a->dx) | reinterpret_cast<uintptr_t>(a->dx2);
    return (u & 15u) == 0 && (a->rows <= 1 || (ld * isz) % 16 == 0);
}

struct BwdCfg {
    int P, nbuf, slice_groups, threads, gamma_smem, nch, chunk_groups;
    long long smem;
};

// Staged geometry: the largest slice of P CTAs, nbuf buffers of two slices,
// and (gamma_smem) the FP32 gamma slice (4 / isz times a slice's bytes).
bool bwd_config(const DeviceInfo &di, long long N, int isz, int P, int req_nbuf, bool gamma_smem, BwdCfg *out) {
    if (P < 1 || P > kMaxCluster || (P & (P - 1)) != 0) return false;
    const long long Gq = N * isz / 16;
    const long long per = (Gq + P - 1) / P;  // groups of the largest slice
    const long long groups = (per + 7) / 8 * 8;  // 128-byte multiples
    if (groups > (1LL << 24)) return false;
    const long long gbytes = gamma_smem ? groups * 16 * (4 / isz) : 0;
    for (int nb = 2; nb >= 1; --nb) {
        if (req_nbuf != 0 && nb != req_nbuf) continue;
        const long long smem = kBwdCtrl + static_cast<long long>(nb) * 2 * groups * 16 + gbytes;
        if (smem <= di.smem_optin) {
            // two buffers: one chunk (the whole next row is in flight anyway).  One buffer: at most
            // kBwdMaxChunks chunks whose size is a multiple of the thread count, so that every thread sums
            // the same groups in the same order as with one chunk (the result does not depend on the
            // buffering)
            long long cgr = groups > 0 ? groups : 1, nch = 1;
            if (nb == 1 && groups > kBwdThreads) {
                const long long per_chunk = (groups + kBwdMaxChunks - 1) / kBwdMaxChunks;
                cgr = (per_chunk + kBwdThreads - 1) / kBwdThreads * kBwdThreads;
                nch = (groups + cgr - 1) / cgr;
            }
            *out = {P, nb, static_cast<int>(groups), kBwdThreads, gamma_smem ? 1 : 0, static_cast<int>(nch),
                    static_cast<int>(cgr), smem};
            return true;
        }
    }
    return false;
}

// gamma is staged in shared memory by the norms when present and 16-byte aligned.
bool stage_gamma(int op, const float *gamma) {
    return (op == BOP_LN || op == BOP_RMS) && gamma != nullptr && (reinterpret_cast<uintptr_t>(gamma) & 15u) == 0;
}

credit_status check_bwd_plan(int dev, const credit_bwd_args *a, const credit_plan_t *p, BwdCfg *cfg, int *maxc) {
    if (p->fill_share != 0.0f || p->retain != 0) return CREDIT_ERR_UNSUPPORTED;
    if (p->threads != 0 && p->threads != kBwdThreads) return CREDIT_ERR_UNSUPPORTED;
    BwdKernels k;
    if (!bwd_kernels(a->op, a->dtype, &k)) return CREDIT_ERR_UNSUPPORTED;
    if (p->path == CREDIT_PATH_TWO_PASS) {
        if (p->ctas_per_row < 1 || p->ctas_per_row > 4096) return CREDIT_ERR_UNSUPPORTED;
        return CREDIT_OK;
    }
    if (p->path != CREDIT_PATH_ONE_CTA && p->path != CREDIT_PATH_CLUSTER) return CREDIT_ERR_UNSUPPORTED;
    const int P = p->path == CREDIT_PATH_ONE_CTA ? 1 : p->cluster_size;
    if (p->path == CREDIT_PATH_CLUSTER && P < 2) return CREDIT_ERR_UNSUPPORTED;
    if (p->ring_chunks < 0 || p->ring_chunks > 2) return CREDIT_ERR_UNSUPPORTED;
    if (!rows_aligned(a)) return CREDIT_ERR_UNSUPPORTED;
    const DeviceInfo *di = device_info(dev);
    if (di == nullptr ||
        !bwd_config(*di, a->cols, dtype_size(a->dtype), P, p->ring_chunks, stage_gamma(a->op, a->gamma), cfg))
        return CREDIT_ERR_UNSUPPORTED;
    const credit_status st = prepare_staged_kernel(dev, k.staged);
    if (st != CREDIT_OK) return st;
    *maxc = staged_max_clusters(dev, k.staged, P, cfg->threads, cfg->smem, false);
    return *maxc > 0 ? CREDIT_OK : CREDIT_ERR_UNSUPPORTED;
}

inline bool kPairOp(int op) { return op == BOP_WVAR || op == BOP_PEARSON; }

credit_status plan_bwd_for(int dev, int op, long long cols, int dtype, credit_plan_t *out) {
    std::memset(out, 0, sizeof(*out));
    out->source = 3;
    out->threads = kBwdThreads;
    const int isz = dtype_size(dtype);
    const DeviceInfo *di = dev >= 0 ? device_info(dev) : nullptr;
    if (di != nullptr && cols * isz > kBwdFusedMaxBytes) {
        BwdKernels k;
        if (!bwd_kernels(op, dtype, &k)) return CREDIT_ERR_UNSUPPORTED;
        const bool merge_heavy = op == BOP_SMLOGITS || op == BOP_XENT || kPairOp(op);
        if (merge_heavy) {
            // the logits ops carry a per-row merge of (max, sum, dot) states, the pair ops Chan merges of
            // centred moments, whose cost and exchange latency grow with P: staged only while a CTA's slice is
            // at most 64 KiB per array and P <= 4 (measured: P = 4 beats two-pass at 64K FP32 columns, P = 8
            // and 16 lose at 128K), either buffering
            for (int P = 1; P <= 4; P *= 2) {
                BwdCfg cfg;
                if (cols * isz > 65536LL * P) continue;
                if (!bwd_config(*di, cols, isz, P, 0, false, &cfg)) continue;
                if (prepare_staged_kernel(dev, k.staged) != CREDIT_OK) continue;
                if (staged_max_clusters(dev, k.staged, P, cfg.threads, cfg.smem, false) <= 0) continue;
                out->path = P == 1 ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
                out->cluster_size = P;
                out->ctas_per_row = P;
                out->ring_chunks = cfg.nbuf;
                out->smem_bytes = cfg.smem;
                return CREDIT_OK;
            }
        }
        // double-buffered staging only: a single buffer leaves the copies of the next row unoverlapped, which
        // measured no faster than the global-reread path
        for (int P = 1; P <= kMaxCluster && !merge_heavy; P *= 2) {
            BwdCfg cfg;
            if (!bwd_config(*di, cols, isz, P, 2, op == BOP_LN || op == BOP_RMS, &cfg)) continue;
            if (prepare_staged_kernel(dev, k.staged) != CREDIT_OK) continue;
            if (staged_max_clusters(dev, k.staged, P, cfg.threads, cfg.smem, false) <= 0) continue;
            out->path = P == 1 ? CREDIT_PATH_ONE_CTA : CREDIT_PATH_CLUSTER;
            out->cluster_size = P;
            out->ctas_per_row = P;
            out->ring_chunks = cfg.nbuf;
            out->smem_bytes = cfg.smem;
            return CREDIT_OK;
        }
    }
    long long g = cols * isz / (256LL << 10);
    out->path = CREDIT_PATH_TWO_PASS;
    out->cluster_size = 1;
    out->ctas_per_row = static_cast<int>(g < 1 ? 1 : (g > 8 ? 8 : g));
    return CREDIT_OK;
}

BwdArgs make_bwd_args(const credit_bwd_args *a, unsigned *err, float *ws) {
    BwdArgs r{};
    r.a = static_cast<const unsigned char *>(a->a);
    r.dy = static_cast<const unsigned char *>(a->dy);
    r.dx = static_cast<unsigned char *>(a->dx);
    r.dx2 = static_cast<unsigned char *>(a->dx2);
    r.rows = a->rows;
    r.cols = a->cols;
    r.ld = a->ld ? a->ld : a->cols;
    r.gamma = a->gamma;
    r.mean = a->mean;
    r.rstd = a->rstd;
    r.scale = a->scale;
    r.err = err;
    r.ws = ws;
    return r;
}

credit_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return CREDIT_OK;
    if (std::getenv("CREDIT_LOG")) std::fprintf(stderr, "credit: CUDA error %s\n", cudaGetErrorString(e));
    return CREDIT_ERR_CUDA;
}

}  // namespace
}  // namespace credit

using namespace credit;

extern "C" {

credit_status credit_plan_bwd(int32_t op, int64_t rows, int64_t cols, credit_dtype dtype, credit_plan_t *out) {
    if (out == nullptr || op < BOP_SOFTMAX || op > BOP_PEARSON || rows < 0 || cols <= 0) return CREDIT_ERR_INVALID_ARG;
    if (dtype != CREDIT_F32 && dtype != CREDIT_BF16) return CREDIT_ERR_UNSUPPORTED;
    int dev = 0;
    const credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    return plan_bwd_for(dev, op, cols, dtype, out);
}

credit_status credit_bwd_plan_check(const credit_bwd_args *args, const credit_plan_t *plan) {
    credit_status st = validate_bwd(args);
    if (st != CREDIT_OK) return st;
    if (plan == nullptr) return CREDIT_ERR_INVALID_ARG;
    int dev = 0;
    if ((st = ensure_init(&dev, nullptr)) != CREDIT_OK) return st;
    BwdCfg cfg;
    int maxc = 0;
    return check_bwd_plan(dev, args, plan, &cfg, &maxc);
}

credit_status credit_run_bwd(const credit_bwd_args *args, const credit_plan_t *plan, cudaStream_t stream) {
    credit_status st = validate_bwd(args);
    if (st != CREDIT_OK) return st;
    if (args->rows == 0) return CREDIT_OK;
    int dev = 0;
    if ((st = ensure_init(&dev, stream)) != CREDIT_OK) return st;
    credit_plan_t chosen;
    if (plan) {
        chosen = *plan;
    } else {
        if ((st = plan_bwd_for(dev, args->op, args->cols, args->dtype, &chosen)) != CREDIT_OK) return st;
        if (chosen.path != CREDIT_PATH_TWO_PASS && !rows_aligned(args)) {  // staged paths need aligned rows
            chosen.path = CREDIT_PATH_TWO_PASS;
            chosen.cluster_size = 1;
            long long g = args->cols * dtype_size(args->dtype) / (256LL << 10);
            chosen.ctas_per_row = static_cast<int>(g < 1 ? 1 : (g > 8 ? 8 : g));
            chosen.ring_chunks = 0;
        }
    }
    BwdCfg cfg{};
    int maxc = 0;
    if ((st = check_bwd_plan(dev, args, &chosen, &cfg, &maxc)) != CREDIT_OK) return st;
    BwdKernels k;
    bwd_kernels(args->op, args->dtype, &k);
    size_t ws_floats = 0;
    float *ws = device_workspace(dev, &ws_floats);
    BwdArgs base = make_bwd_args(args, device_error_word(dev), ws);
    const long long rows = args->rows;
    cudaError_t e;

    if (chosen.path != CREDIT_PATH_TWO_PASS) {
        const long long ncl = rows < maxc ? rows : maxc;
        BwdArgs r = base;
        r.nbuf = cfg.nbuf;
        r.slice_groups = cfg.slice_groups;
        r.gamma_smem = cfg.gamma_smem;
        r.nch = cfg.nch;
        r.chunk_groups = cfg.chunk_groups;
        void *kargs[] = {&r};
        e = launch_kernel(k.staged, dim3(static_cast<unsigned>(cfg.P * ncl)), dim3(cfg.threads),
                          static_cast<size_t>(cfg.smem), cfg.P, stream, kargs);
        if (e != cudaSuccess) return cuda_st(e);
        g_launch_count.fetch_add(1);
        return CREDIT_OK;
    }
    const int G = chosen.ctas_per_row;
    const size_t rec = (args->op == BOP_SMLOGITS || args->op == BOP_XENT) ? 4
                       : (args->op == BOP_WVAR || args->op == BOP_PEARSON) ? 8 : 2;  // floats per partial
    const long long cap = G == 1 ? 0x7FFFFFFFLL : static_cast<long long>(ws_floats / (static_cast<size_t>(G) * rec));
    const long long max_rows = cap < 0x7FFFFFFFLL / G ? cap : 0x7FFFFFFFLL / G;
    if (max_rows < 1) return CREDIT_ERR_UNSUPPORTED;
    for (long long r0 = 0; r0 < rows; r0 += max_rows) {
        const long long n = rows - r0 < max_rows ? rows - r0 : max_rows;
        BwdArgs r = base;
        r.row0 = r0;
        r.G = G;
        void *kargs[] = {&r};
        if (G == 1) {
            e = launch_kernel(k.fused, dim3(static_cast<unsigned>(n)), dim3(kBwdThreads), 0, 1, stream, kargs);
            if (e != cudaSuccess) return cuda_st(e);
            g_launch_count.fetch_add(1);
            continue;
        }
        const dim3 grid(static_cast<unsigned>(G * n));
        e = launch_kernel(k.stats, grid, dim3(kBwdThreads), 0, 1, stream, kargs);
        if (e != cudaSuccess) return cuda_st(e);
        g_launch_count.fetch_add(1);
        e = launch_kernel(k.apply, grid, dim3(kBwdThreads), 0, 1, stream, kargs);
        if (e != cudaSuccess) return cuda_st(e);
        g_launch_count.fetch_add(1);
    }
    return CREDIT_OK;
}

}  // extern "C"
