// credit_control.cu -- the structural screen of the profitability model and
// the negative controls it rejects (CREDIT Sec. III-D, last paragraph;
// Sec. IV-C, negative controls).
//
// Before any clustered variant is generated, an op's dataflow decides
// whether the cluster path can pay at all.  The paper rejects three cases by
// construction, because growing the row width N cannot help them:
//   - nothing to reuse: no reduction stage whose statistics every element of
//     the row needs (an elementwise op, a stencil), or a reduction whose
//     output is the statistic itself (log-sum-exp): the global-reread
//     baseline rereads nothing, b_reread = 0, so T_save = 0 in Eq. 9;
//   - ordered dependencies: the result a CTA applies depends on the CTAs
//     before it in order (a scan's carries), so the barrier count K grows
//     with P instead of staying 2L;
//   - remote state that grows with N (selection, top-k, medians): what the
//     CTAs exchange is data, not the compact sum of q_l statistics of Eq. 6.
//
// The two executable controls run on the non-DSMEM global-memory path:
//   k_ctrl_scan     row-wise inclusive prefix sum, one CTA per row, one read
//                   and one write of every element: tiles of 4 elements per
//                   thread, shuffle scans of the thread and warp totals, and
//                   a carry across tiles kept with Kahan compensation.
//   k_ctrl_stencil  row-wise stencil of radius r <= 8 with zero padding at the
//                   row ends; a CTA stages the inputs of 4096 outputs in
//                   shared memory once and every thread writes 16 of them.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_prim.cuh"

namespace credit {
extern std::atomic<long long> g_launch_count;
}

using namespace credit;

namespace {

constexpr int kScanThreads = 512;
constexpr int kStencilThreads = 256;
constexpr int kStencilTile = 4096;  // outputs per CTA
constexpr int kMaxRadius = 8;

__device__ __forceinline__ float warp_inclusive_scan(float v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_ctrl_scan(const float *__restrict__ in, float *__restrict__ out,
                                                            long long cols, long long ld_in, long long ld_out) {
    __shared__ float wsum[32];
    const long long row = blockIdx.x;
    const float *x = in + row * ld_in;
    float *y = out + row * ld_out;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0;
    float carry = 0.0f, comp = 0.0f;  // running total of the tiles before this one (Kahan)
    for (long long t0 = 0; t0 < cols; t0 += 4LL * blockDim.x) {
        const long long i = t0 + 4LL * tid;
        float v[4];
        if (vec && i + 3 < cols) {
            const float4 q = *reinterpret_cast<const float4 *>(x + i);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = i + k < cols ? x[i + k] : 0.0f;
        }
        v[1] += v[0];
        v[2] += v[1];
        v[3] += v[2];
        const float tsum = v[3];
        const float ws = warp_inclusive_scan(tsum);
        if (lane == 31) wsum[wid] = ws;
        __syncthreads();
        if (wid == 0) {
            const float s = warp_inclusive_scan(lane < nw ? wsum[lane] : 0.0f);
            if (lane < nw) wsum[lane] = s;
        }
        __syncthreads();
        const float base = (ws - tsum) + (wid > 0 ? wsum[wid - 1] : 0.0f);  // exclusive prefix within the tile
        const float tile_total = wsum[nw - 1];
        __syncthreads();  // wsum is rewritten by the next tile
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = carry + (base + v[k]);
        if (vec && i + 3 < cols) {
            *reinterpret_cast<float4 *>(y + i) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i + k < cols) y[i + k] = o[k];
        }
        const float yk = tile_total - comp;  // carry += tile_total, compensated
        const float t = carry + yk;
        comp = (t - carry) - yk;
        carry = t;
    }
}

// One CTA per tile of kStencilTile outputs of a row: the inputs the tile
// needs (kStencilTile + 2r, widened to 16-byte address boundaries) are loaded
// once into shared memory -- every thread issues all of its float4 loads
// before storing any, so a CTA keeps 16 KiB in flight -- float4 where the
// whole vector lies inside the row, zero outside it.  Thread t then computes
// outputs t, t + T, t + 2T, ... of the tile: a warp's shared reads and global
// stores are consecutive.
__global__ void __launch_bounds__(kStencilThreads) k_ctrl_stencil(const float *__restrict__ in,
                                                                  float *__restrict__ out, long long cols,
                                                                  long long ld_in, long long ld_out,
                                                                  const float *__restrict__ weights, int r) {
    __shared__ float w[2 * kMaxRadius + 1];
    __shared__ __align__(16) float tile[kStencilTile + 2 * kMaxRadius + 8];
    constexpr int kQ = (kStencilTile + 2 * kMaxRadius + 8) / 4 / kStencilThreads + 1;  // float4 loads per thread
    const int tid = threadIdx.x;
    if (tid < 2 * r + 1) w[tid] = weights[tid];
    const long long row = blockIdx.y;
    const float *x = in + row * ld_in;
    float *y = out + row * ld_out;
    const long long t0 = static_cast<long long>(blockIdx.x) * kStencilTile;
    const long long need_lo = t0 - r, need_hi = min(t0 + kStencilTile, cols) + r;
    // first index at or below need_lo whose address is 16-byte aligned (x is 4-byte aligned)
    const long long lo = need_lo - static_cast<long long>((reinterpret_cast<uintptr_t>(x) / 4 + need_lo) & 3);
    const int nq = static_cast<int>((need_hi - lo + 3) / 4);
    float4 v[kQ];
#pragma unroll
    for (int u = 0; u < kQ; ++u) {
        const int q = tid + u * kStencilThreads;
        const long long j = lo + 4LL * q;
        if (q >= nq) {
            v[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else if (j >= 0 && j + 3 < cols) {
            v[u] = *reinterpret_cast<const float4 *>(x + j);
        } else {
            v[u].x = (j >= 0 && j < cols) ? x[j] : 0.0f;
            v[u].y = (j + 1 >= 0 && j + 1 < cols) ? x[j + 1] : 0.0f;
            v[u].z = (j + 2 >= 0 && j + 2 < cols) ? x[j + 2] : 0.0f;
            v[u].w = (j + 3 >= 0 && j + 3 < cols) ? x[j + 3] : 0.0f;
        }
    }
#pragma unroll
    for (int u = 0; u < kQ; ++u) {
        const int q = tid + u * kStencilThreads;
        if (q < nq) *reinterpret_cast<float4 *>(tile + 4 * q) = v[u];
    }
    __syncthreads();
    const int off = static_cast<int>(t0 - r - lo);  // tile index of input t0 - r
    const int n_out = static_cast<int>(min(static_cast<long long>(kStencilTile), cols - t0));
    for (int o = tid; o < n_out; o += kStencilThreads) {
        float acc = 0.0f;
        for (int m = 0; m <= 2 * r; ++m) acc = fmaf(w[m], tile[off + o + m], acc);
        y[t0 + o] = acc;
    }
}

}  // namespace

extern "C" {

credit_status credit_dataflow_of(int32_t op, credit_dtype in_dtype, credit_dataflow *out) {
    if (out == nullptr || in_dtype < 0 || in_dtype > 2) return CREDIT_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    const double isz = dtype_size(in_dtype);
    switch (op) {
    case CREDIT_OP_SOFTMAX:       // (m, s), h applied to every element
    case CREDIT_OP_LAYERNORM:     // (mean, M2)
        *out = {1, 0, 2.0, isz, 0.0};
        return CREDIT_OK;
    case CREDIT_OP_RMSNORM:       // sum of squares
    case CREDIT_OP_QUANT_INT8:    // amax
        *out = {1, 0, 1.0, isz, 0.0};
        return CREDIT_OK;
    case CREDIT_OP_LOGSUMEXP:     // one pass; the statistic is the output: nothing is reread
        *out = {1, 0, 2.0, 0.0, 0.0};
        return CREDIT_OK;
    case CREDIT_OP_SCAN:          // a carry per CTA, but CTA c needs the carries of CTAs 0..c-1 in order
        *out = {1, 1, 1.0, isz, 0.0};
        return CREDIT_OK;
    case CREDIT_OP_STENCIL:       // no reduction stage: neighbours' halo elements, not statistics
        *out = {0, 0, 0.0, 0.0, 0.0};
        return CREDIT_OK;
    case CREDIT_OP_SELECT:        // top-k / median: the candidates exchanged are a share of the slice itself
        *out = {1, 0, 0.0, isz, isz};
        return CREDIT_OK;
    default: return CREDIT_ERR_INVALID_ARG;
    }
}

credit_status credit_screen(const credit_dataflow *d, int32_t P, int32_t *verdict, int32_t *K) {
    if (d == nullptr || verdict == nullptr || P < 1 || P > 16 || d->stages < 0) return CREDIT_ERR_INVALID_ARG;
    // barrier count per row: K = 2L for the push all-gather of Eq. 5-6; a chain of ordered carries adds
    // one dependent exchange per CTA boundary of every stage
    if (K) *K = d->ordered ? 2 * d->stages * (P > 1 ? P - 1 : 1) : 2 * d->stages;
    if (d->stages == 0 || !(d->b_reread > 0.0)) *verdict = CREDIT_SCREEN_NO_REUSE;
    else if (d->ordered) *verdict = CREDIT_SCREEN_ORDERED;
    else if (d->remote_bytes_per_elem > 0.0) *verdict = CREDIT_SCREEN_REMOTE_STATE;
    else *verdict = CREDIT_SCREEN_CANDIDATE;
    return CREDIT_OK;
}

credit_status credit_plan_control(int32_t op, int64_t rows, int64_t cols, credit_plan_t *out, int32_t *verdict) {
    if (out == nullptr || rows < 0 || cols <= 0 || (op != CREDIT_OP_SCAN && op != CREDIT_OP_STENCIL))
        return CREDIT_ERR_INVALID_ARG;
    credit_dataflow d;
    credit_dataflow_of(op, CREDIT_F32, &d);
    int32_t v = 0;
    credit_screen(&d, 16, &v, nullptr);
    std::memset(out, 0, sizeof(*out));
    out->path = CREDIT_PATH_TWO_PASS;  // the non-DSMEM global-memory path
    out->cluster_size = 1;
    out->ctas_per_row = op == CREDIT_OP_SCAN ? 1 : static_cast<int32_t>((cols + kStencilTile - 1) / kStencilTile);
    out->threads = op == CREDIT_OP_SCAN ? kScanThreads : kStencilThreads;
    out->source = 3;
    if (verdict) *verdict = v;
    return CREDIT_OK;
}

credit_status credit_run_control(int32_t op, const float *in, float *out, int64_t rows, int64_t cols, int64_t ld_in,
                                 int64_t ld_out, const float *weights, int32_t radius, cudaStream_t stream) {
    if (op != CREDIT_OP_SCAN && op != CREDIT_OP_STENCIL) return CREDIT_ERR_INVALID_ARG;
    if (rows < 0 || cols <= 0 || ld_in < 0 || ld_out < 0 || (ld_in && ld_in < cols) || (ld_out && ld_out < cols))
        return CREDIT_ERR_INVALID_ARG;
    if (rows == 0) return CREDIT_OK;
    if (in == nullptr || out == nullptr || (reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % 4)
        return CREDIT_ERR_INVALID_ARG;
    if (op == CREDIT_OP_STENCIL && (weights == nullptr || radius < 0 || radius > kMaxRadius))
        return CREDIT_ERR_INVALID_ARG;
    if (op == CREDIT_OP_STENCIL && in == out) return CREDIT_ERR_INVALID_ARG;  // it reads neighbours it overwrites
    if (rows > 0x7FFFFFFFLL) return CREDIT_ERR_UNSUPPORTED;
    const long long li = ld_in ? ld_in : cols, lo = ld_out ? ld_out : cols;
    cudaError_t e;
    if (op == CREDIT_OP_SCAN) {
        k_ctrl_scan<<<static_cast<unsigned>(rows), kScanThreads, 0, stream>>>(in, out, cols, li, lo);
        e = cudaGetLastError();
    } else {
        const long long bx = (cols + kStencilTile - 1) / kStencilTile;
        if (bx > 0x7FFFFFFFLL || rows > 65535) return CREDIT_ERR_UNSUPPORTED;
        k_ctrl_stencil<<<dim3(static_cast<unsigned>(bx), static_cast<unsigned>(rows)), kStencilThreads, 0, stream>>>(
            in, out, cols, li, lo, weights, radius);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    g_launch_count.fetch_add(1);
    return CREDIT_OK;
}

}  // extern "C"
