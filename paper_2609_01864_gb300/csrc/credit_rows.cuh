// credit_rows.cuh -- row kernels of the reduction-reuse ops (CREDIT Sec. III).
//
// Op model (Eq. 1): a row of N elements is reduced to q scalar statistics per
// stage, then every element is mapped through h.
//   softmax    stage 1: q = 2, (m, s): m = max x, s = sum exp(x - m)
//              h(x) = exp(x - m) / s
//   logsumexp  the softmax statistics; the row's output is m + ln s (no h)
//   layernorm  stage 1: q = 2, (mean, M2) merged with Chan's formula
//              h(x) = (x - mean) * rsqrt(M2 / N + eps) * gamma + beta
//   rmsnorm    stage 1: q = 1, sum x^2;  h(x) = x * rsqrt(sum/N + eps) * gamma
//   FP8 output of layernorm / rmsnorm adds stage 2: q = 1, amax |h(x)|, and
//   writes codes h(x) * 448 / amax with the row scale amax / 448.  Softmax
//   needs no extra stage: its amax is 1 / s in closed form.
//   int8       stage 1: q = 1, amax |x| (merged by max);  s = amax / 127
//   quantise   (1 for an all-zero row), h(x) = clamp(rint(x / s), +-127)
//              with both quotients correctly rounded in FP32; the row's
//              scale s goes to out_scale.
//
// Slicing (Eq. 2).  A row is cut on the 16-byte grid of its own address: the
// elements before the first 16-byte boundary (the "head", < 16 bytes) belong
// to CTA 0, the elements after the last full 16-byte group (the "tail") to CTA
// P-1, and the G full groups in between are split evenly, CTA c taking groups
// [G*c/P, G*(c+1)/P).  The same rule with P -> ctas_per_row slices rows in
// the split-row two-pass path.
//
// Kernels
//   k_ring       a cluster of P CTAs per row (P = 1: the one-CTA path),
//                persistent over rows.  Each CTA stages its slice into its
//                own shared memory with cp.async.bulk through a ring of
//                chunks (the first reduction sweep overlaps the copy, the
//                next row's copy overlaps this row's writes), reduces
//                locally (threads -> warp shuffles -> shared memory), pushes
//                its partials into every peer's slot array over DSMEM (Eq. 5:
//                one of the first P threads per destination), combines the P
//                local slots in fixed order c = 0..P-1 (so every CTA holds
//                bit-identical statistics), and writes its output segment
//                from shared memory (Sec. III-C, "reuse").
//   k_tp_fused   the global-reread baseline with one CTA per row: a
//                statistics sweep over HBM, then a sweep that rereads the row
//                (Sec. IV-A; Eq. 4 with b_reread = input bytes).
//   k_tp_stats / k_tp_amax / k_tp_apply / k_tp_lse_final
//                the same baseline with G CTAs per row: partials go to a
//                device workspace and the next launch is the barrier; no
//                kernel ever waits on another CTA.
#pragma once

#include <type_traits>

#include "credit_prim.cuh"

namespace credit {

struct RowArgs {
    const unsigned char *in;
    unsigned char *out;
    long long rows, cols, ld_in, ld_out;  // strides in elements
    const float *in_scale;                // FP8 input: per-row scale
    float *out_scale;                     // FP8 output: per-row scale
    const float *gamma, *beta;
    float eps;
    unsigned *err;                        // device error word
    float *ws;                            // two-pass partials [row - row0][G][4]
    int G;                                // CTAs per row of the two-pass path
    int chunk_bytes;                      // ring kernel: bytes per staged chunk
    int ring;                             // ring kernel: chunk slots
    int reducers;                         // ring kernel: reducer threads (multiple of 32)
    int affine;                           // ring kernel: gamma/beta ring slots (0 = direct loads)
    int affine_resident;                  // 1: the slots hold the whole slice's gamma/beta, loaded once
    unsigned long long *trace;            // optional phase timestamps (see credit_set_trace)
    int trace_rows;                       // rows recorded per traced CTA
    long long row0;                       // first row of this launch
    unsigned long long wait_ns;           // limit of the reducers' chunk waits (ns; 0 = kWaitLimitNs)
    int test_extra_tx;                    // test only: extra bytes the first chunk's barrier expects (0)
};

constexpr int kMaxCluster = 16;
constexpr int kMaxChunkBytes = 16384;  // default (and largest) staged chunk

// Position of a role in a ring of n slots that it uses in order: the slot of
// its next use and the number of completed laps (the phase parity an
// mbarrier of that slot is at).  Kept incrementally, so the per-chunk loops
// never divide a running 64-bit chunk count by the ring size.
struct RingPos {
    int slot = 0, n = 1;
    uint32_t lap = 0;
    __device__ __forceinline__ explicit RingPos(int slots) : n(slots) {}
    __device__ __forceinline__ void next() {
        if (++slot == n) {
            slot = 0;
            ++lap;
        }
    }
    // parity of this lap's phase (a consumer waiting for the slot to fill)
    __device__ __forceinline__ uint32_t parity() const { return lap & 1u; }
    // parity of the previous lap's release (a producer reusing the slot)
    __device__ __forceinline__ uint32_t prev_parity() const { return (lap - 1u) & 1u; }
    // the position k uses later (k >= 0; one subtraction per lap crossed)
    __device__ __forceinline__ RingPos at(int k) const {
        RingPos r(*this);
        r.slot += k;
        while (r.slot >= r.n) {
            r.slot -= r.n;
            ++r.lap;
        }
        return r;
    }
    __device__ __forceinline__ void advance(int k) { *this = at(k); }
};

struct RowSlice {
    long long h0;          // head elements (rank 0)
    long long G;           // full 16-byte groups after the head
    long long t0;          // tail elements (rank P-1)
    long long g_lo, g_hi;  // this CTA's groups
};

// floor(G * k / P) for 0 <= k <= P (P = cluster size, or CTAs per row of the
// split two-pass path, up to 4096): 32-bit unsigned arithmetic when G * P, and
// so every G * k, fits in 32 bits (the common case; exact, so identical to
// the 64-bit form), else 64-bit.
__host__ __device__ __forceinline__ long long group_split(long long G, int k, int P) {
    if (static_cast<unsigned long long>(G) * static_cast<unsigned>(P) <= 0xFFFFFFFFull)
        return static_cast<long long>(static_cast<uint32_t>(G) * static_cast<uint32_t>(k) / static_cast<uint32_t>(P));
    return G * k / P;
}

__host__ __device__ __forceinline__ RowSlice make_slice(uintptr_t row_addr, long long N, int isz, int P, int c) {
    const int V = 16 / isz;
    const long long mis = static_cast<long long>(row_addr & 15u);
    long long h0 = mis ? (16 - mis) / isz : 0;
    if (h0 > N) h0 = N;
    const long long rest = N - h0;
    RowSlice s;
    s.h0 = h0;
    s.G = rest / V;
    s.t0 = rest - s.G * V;
    s.g_lo = group_split(s.G, c, P);
    s.g_hi = group_split(s.G, c + 1, P);
    return s;
}

// Elements owned by CTA c (of P) for a row with h0 / G / t0.
__host__ __device__ __forceinline__ long long slice_count(const RowSlice &s, int V, int P, int c) {
    const long long lo = group_split(s.G, c, P), hi = group_split(s.G, c + 1, P);
    return (hi - lo) * V + (c == 0 ? s.h0 : 0) + (c == P - 1 ? s.t0 : 0);
}

// ------------------------------------------------------------------ stats
// Per-CTA partials are two floats for every op:
//   softmax / lse: (m_c, s_c)   layernorm: (mean_c, M2_c)   rmsnorm: (ss_c, 0)
// Row statistics after the combine:
//   softmax / lse: (M, S)       layernorm: (mean, rstd)     rmsnorm: (rstd, 0)
struct Stats {
    float a, b;
};

// Combine partials p[c*stride + 0/1], c = 0..P-1, in fixed order.
template <int OP>
__device__ __forceinline__ Stats combine_partials(const float *p, int stride, int P, const RowSlice &s, int V,
                                                  long long N, float eps) {
    Stats st;
    if constexpr (OP == OP_SOFTMAX || OP == OP_LSE) {
        float M = -INFINITY;
        for (int c = 0; c < P; ++c) M = fmaxf(M, p[c * stride]);
        float S = 0.0f;
        for (int c = 0; c < P; ++c) {
            const float sc = p[c * stride + 1];
            if (sc > 0.0f) S += sc * exp_fast(p[c * stride] - M);
        }
        st.a = M;
        st.b = S;
    } else if constexpr (OP == OP_LN) {
        float n = 0.0f, mu = 0.0f, m2 = 0.0f;
        for (int c = 0; c < P; ++c) {
            const float nb = static_cast<float>(slice_count(s, V, P, c));
            if (nb == 0.0f) continue;
            const float nn = n + nb;
            const float d = p[c * stride] - mu;
            mu += d * (nb / nn);
            m2 += p[c * stride + 1] + d * d * (n * nb / nn);
            n = nn;
        }
        st.a = mu;
        st.b = rsqrtf(m2 / static_cast<float>(N) + eps);
    } else if constexpr (OP == OP_Q8) {
        float am = 0.0f;
        for (int c = 0; c < P; ++c) am = fmaxf(am, p[c * stride]);
        st.a = am > 0.0f ? __fdiv_rn(am, 127.0f) : 1.0f;  // the row scale
        st.b = __frcp_rn(st.a);                              // its correctly rounded reciprocal
    } else {
        float ss = 0.0f;
        for (int c = 0; c < P; ++c) ss += p[c * stride];
        st.a = rsqrtf(ss / static_cast<float>(N) + eps);
        st.b = 0.0f;
    }
    return st;
}

// h(x) for LayerNorm / RMSNorm.
template <int OP>
__device__ __forceinline__ float norm_h(float x, const Stats &st, float g, float b) {
    if constexpr (OP == OP_LN) return (x - st.a) * st.b * g + b;
    else return x * st.a * g;
}

template <int V>
__device__ __forceinline__ void load_affine(const float *p, long long i0, bool vec, float dflt, float (&v)[V]) {
    if (p == nullptr) {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = dflt;
    } else if (vec) {
#pragma unroll
        for (int k = 0; k < V / 4; ++k) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(p + i0) + k);
            v[4 * k] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = __ldg(p + i0 + k);
    }
}

// SV affine values from the shared-memory affine ring (p == nullptr: dflt).
template <int SV>
__device__ __forceinline__ void load_affine_smem(const float *p, int off, float dflt, float (&v)[SV]) {
    if (p == nullptr) {
#pragma unroll
        for (int k = 0; k < SV; ++k) v[k] = dflt;
    } else {
        const uint32_t base = smem_addr(p + off);
#pragma unroll
        for (int k = 0; k < SV / 4; ++k)
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(v[4 * k]), "=f"(v[4 * k + 1]), "=f"(v[4 * k + 2]), "=f"(v[4 * k + 3])
                         : "r"(base + 16 * k));
    }
}

// N floats from shared memory at p (16-byte aligned), 16 bytes per load.
template <int N>
__device__ __forceinline__ void lds_f32(const float *p, float (&v)[N]) {
    const uint32_t base = smem_addr(p);
#pragma unroll
    for (int k = 0; k < N / 4; ++k)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v[4 * k]), "=f"(v[4 * k + 1]), "=f"(v[4 * k + 2]), "=f"(v[4 * k + 3])
                     : "r"(base + 16 * k));
}

__device__ __forceinline__ void copy_raw(unsigned char *dst, const unsigned char *src, int isz) {
    if (isz == 4) *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(src);
    else if (isz == 2) *reinterpret_cast<uint16_t *>(dst) = *reinterpret_cast<const uint16_t *>(src);
    else *dst = *src;
}

// ======================================================================
// Per-thread streaming statistics (one sweep; used by every path)
// ======================================================================
template <int OP> struct Stream;

// Maximum of N values as a tree (dependency depth log2 N; the same value as any order).
template <int N>
__device__ __forceinline__ float max_of(const float (&f)[N]) {
    if constexpr (N == 1) {
        return f[0];
    } else {
        float h[(N + 1) / 2];
#pragma unroll
        for (int j = 0; j < N / 2; ++j) h[j] = fmaxf(f[2 * j], f[2 * j + 1]);
        if constexpr (N % 2 == 1) h[N / 2] = f[N - 1];
        return max_of(h);
    }
}

template <> struct Stream<OP_SOFTMAX> {  // online (max, sum exp)
    float m = -INFINITY, s = 0.0f;
    __device__ __forceinline__ void raise(float mv) {
        if (mv > m) {
            s *= ex2_ftz((m - mv) * kLog2e);
            m = mv;
        }
    }
    // The terms 2^((f - m) log2 e) of a group (the difference first, so the
    // error does not grow with |m|), two at a time on packed f32x2 ops,
    // subnormal terms flushed (ex2_ftz), summed as a tree.
    template <int V> __device__ __forceinline__ void add(const float (&f)[V]) {
        const float mv = max_of(f);
        if (mv == -INFINITY) return;
        raise(mv);
        if constexpr (V % 4 == 0) {
            float e[V];
#pragma unroll
            for (int j = 0; j < V; j += 2) {
                const float2 t = __fmul2_rn(__fadd2_rn(make_float2(f[j], f[j + 1]), make_float2(-m, -m)),
                                            make_float2(kLog2e, kLog2e));
                e[j] = ex2_ftz(t.x);
                e[j + 1] = ex2_ftz(t.y);
            }
            s += sum_tree<V>(e);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) s += ex2_ftz((f[j] - m) * kLog2e);
        }
    }
    // One 16-byte group of E4M3 codes q of a row whose elements are x = a q
    // (a = |in_scale|; a negative scale has been folded into the codes' sign
    // bits).  The group maximum is taken on the decoded halves (E4M3 is a
    // subset of FP16, and x is increasing in q); each difference x - m is one
    // FMA, a q - m rounded once, two codes per packed op.
    __device__ __forceinline__ void add_e4m3(const uint4 &w, float a) {
        __half2 h[8];
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __half2_raw r0 = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(u[k] & 0xFFFFu), __NV_E4M3);
            __half2_raw r1 = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(u[k] >> 16), __NV_E4M3);
            h[2 * k] = *reinterpret_cast<__half2 *>(&r0);
            h[2 * k + 1] = *reinterpret_cast<__half2 *>(&r1);
        }
        const __half2 mx = __hmax2(__hmax2(__hmax2(h[0], h[1]), __hmax2(h[2], h[3])),
                                   __hmax2(__hmax2(h[4], h[5]), __hmax2(h[6], h[7])));
        raise(fmaxf(__low2float(mx), __high2float(mx)) * a);
        float e[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 t = __fmul2_rn(__ffma2_rn(__half22float2(h[k]), make_float2(a, a), make_float2(-m, -m)),
                                        make_float2(kLog2e, kLog2e));
            e[2 * k] = ex2_ftz(t.x);
            e[2 * k + 1] = ex2_ftz(t.y);
        }
        s += sum_tree<16>(e);
    }
    __device__ __forceinline__ void add1(float x) {
        float f[1] = {x};
        add<1>(f);
    }
    __device__ __forceinline__ void merge(float m2, float s2) {
        if (s2 == 0.0f) return;
        if (s == 0.0f) {
            m = m2;
            s = s2;
            return;
        }
        const float M = fmaxf(m, m2);
        s = s * ex2_ftz((m - M) * kLog2e) + s2 * ex2_ftz((m2 - M) * kLog2e);
        m = M;
    }
    __device__ __forceinline__ float p0() const { return m; }
    __device__ __forceinline__ float p1() const { return s; }
};
template <> struct Stream<OP_LSE> : Stream<OP_SOFTMAX> {};

// Sign bits of 16 E4M3 codes flipped by `neg` (0x80808080 or 0): a row with a
// negative input scale a becomes the row -q with scale |a|.
__device__ __forceinline__ uint4 e4m3_fold_sign(uint4 w, uint32_t neg) {
    return make_uint4(w.x ^ neg, w.y ^ neg, w.z ^ neg, w.w ^ neg);
}
__device__ __forceinline__ uint32_t e4m3_sign_mask(float in_sc) { return in_sc < 0.0f ? 0x80808080u : 0u; }

// One 16-byte group of a row into the op's statistics: E4M3 softmax / log-sum-exp rows on the raw codes
// (Stream::add_e4m3), everything else decoded first.
template <int OP, int TIN>
__device__ __forceinline__ void stream_add_group(Stream<OP> &acc, const uint4 &w, float in_sc) {
    if constexpr (TIN == DT_E4M3 && (OP == OP_SOFTMAX || OP == OP_LSE)) {
        acc.add_e4m3(e4m3_fold_sign(w, e4m3_sign_mask(in_sc)), fabsf(in_sc));
    } else {
        float f[Fmt<TIN>::V];
        decode_group<TIN>(w, f, in_sc);
        acc.add(f);
    }
}

// Softmax output codes of one 16-byte group of E4M3 input codes q (sign folded, x = a q): code =
// 448 exp(x - M) = 2^((a q - M) log2 e + log2 448), two codes per packed op -- the exponent from two
// packed FMAs, rounded to FP16, raised by the packed FP16 SFU op and converted to two E4M3 codes at
// once.  The FP16 rounding of the exponent (|t| < 16: error <= 2^-8) and the SFU's 2^-9.9 move a code's
// value by under 0.5% relative, a small part of an E4M3 step (2^-3 relative).
__device__ __forceinline__ uint4 softmax_e4m3_codes(const uint4 &w, float a, float M) {
    const float c8 = 8.807354922057604f;  // log2 448
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
    uint32_t o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t code2[2];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            __half2_raw r =
                __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>((u[k] >> (16 * hh)) & 0xFFFFu), __NV_E4M3);
            const float2 d = __ffma2_rn(__half22float2(*reinterpret_cast<__half2 *>(&r)), make_float2(a, a),
                                        make_float2(-M, -M));
            const float2 t = __ffma2_rn(d, make_float2(kLog2e, kLog2e), make_float2(c8, c8));
            const __half2 e = ex2_h2(__float22half2_rn(t));
            code2[hh] = __nv_cvt_halfraw2_to_fp8x2(*reinterpret_cast<const __half2_raw *>(&e), __NV_SATFINITE,
                                                   __NV_E4M3);
        }
        o[k] = (code2[0] & 0xFFFFu) | (code2[1] << 16);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

// LayerNorm statistics in one sweep: each thread accumulates sums about a
// shift K (its first element), s1 = sum (x - K), s2 = sum (x - K)^2, and
// converts them once to (n, mean, M2) = (n, K + s1/n, s2 - s1^2/n) before the
// CTA merge (Chan's formula).  The shift is a sample of the thread's own
// data, so the cancellation in s2 - s1^2/n stays small.
template <> struct Stream<OP_LN> {
    float n = 0.0f, mu = 0.0f, m2 = 0.0f;  // merged form (after finish())
    float K = 0.0f, s1 = 0.0f, s2 = 0.0f;
    bool has = false;
    // Chan's merge of (nb, mb, m2b) into this state.  The two quotients use
    // one SFU reciprocal of the merged count (a few ulp each instead of two
    // IEEE divisions on the reduction's critical path).
    __device__ __forceinline__ void merge3(float nb, float mb, float m2b) {
        if (nb == 0.0f) return;
        if (n == 0.0f) {
            n = nb;
            mu = mb;
            m2 = m2b;
            return;
        }
        const float nn = n + nb;
        const float r = rcp_approx(nn);
        const float d = mb - mu;
        const float wb = nb * r;
        mu += d * wb;
        m2 += m2b + d * d * (n * wb);
        n = nn;
    }
    template <int V> __device__ __forceinline__ void add(const float (&f)[V]) {
        if (!has) {
            K = f[0];
            has = true;
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const float d = f[j] - K;
            s1 += d;
            s2 = fmaf(d, d, s2);
        }
        n += static_cast<float>(V);
    }
    __device__ __forceinline__ void add1(float x) {
        float f[1] = {x};
        add<1>(f);
    }
    // (n, K, s1, s2) -> (n, mean, M2); call once before merging
    __device__ __forceinline__ void finish() {
        if (n > 0.0f) {
            const float q = s1 * rcp_approx(n);
            mu = K + q;
            m2 = fmaxf(s2 - s1 * q, 0.0f);
        }
    }
};

template <> struct Stream<OP_RMS> {
    float ss = 0.0f;
    template <int V> __device__ __forceinline__ void add(const float (&f)[V]) {
#pragma unroll
        for (int j = 0; j < V; ++j) ss = fmaf(f[j], f[j], ss);
    }
    __device__ __forceinline__ void add1(float x) { ss = fmaf(x, x, ss); }
};

template <> struct Stream<OP_Q8> {  // amax |x|: exact, so every merge order gives the same value
    float am = 0.0f;
    template <int V> __device__ __forceinline__ void add(const float (&f)[V]) {
#pragma unroll
        for (int j = 0; j < V; ++j) am = fmaxf(am, fabsf(f[j]));
    }
    __device__ __forceinline__ void add1(float x) { am = fmaxf(am, fabsf(x)); }
};

// ======================================================================
// Ring kernel: the cluster path (P > 1) and the one-CTA path (P == 1).
//
// Persistent: grid = nclusters * P CTAs with cluster dims (P, 1, 1); cluster
// k handles rows k, k + nclusters, ...  Three warp roles per CTA:
//   producer (last warp; lane 0)  streams row slices into a ring of `ring`
//            chunk slots of `chunk_bytes` with cp.async.bulk.  The slices of
//            successive rows form one chunk sequence j = 0, 1, ...; chunk j
//            lives in slot j % ring; full[s] completes when it has landed
//            (transaction bytes), empty[s] when every writer warp is done
//            with it.
//   reducers (first `reducers` threads)  sweep each slice as its chunks land,
//            reduce within the CTA (warp shuffles, then shared memory),
//            exchange partials with the cluster (Eq. 5), combine them, and
//            publish the row statistics in a double-buffered stats slot.
//   writers  (the threads in between)  wait for a row's statistics, apply h
//            to the retained slice (the reuse pass) and store the output
//            segment, releasing each chunk to the producer.
//   For LayerNorm / RMSNorm with gamma / beta, producer lane 1 stages the
//   gamma / beta segment of each chunk in an affine ring, so the reuse pass
//   reads only shared memory.  A persistent CTA handles the same columns for
//   every row, so when the ring has one slot per chunk of the slice the
//   segments are loaded once per launch and stay resident; otherwise they
//   stream just ahead of the writers (served from L2).
// So row r is written while row r+1 is being reduced and exchanged and
// row r+2 is streaming in: the cluster exchange and the reductions leave the
// output stream busy.  A slice needs ceil(body / chunk_bytes) <= ring slots
// (Eq. 3).
//
// Exchange (Eq. 5): reducer thread t < P pushes the CTA's partials into slot
// [c] of peer t with st.async, which completes on the peer's exchange
// mbarrier; each CTA waits (bounded) on its own exchange mbarrier for the
// P - 1 remote pushes, then combines its P local slots in fixed order
// c = 0..P-1, so every CTA holds bit-identical statistics.  Slot arrays and
// exchange mbarriers are double-buffered by row parity, so a peer can run one
// row ahead without overwriting partials still being read.  One cluster
// barrier at the start (every CTA's mbarriers are initialised before any
// remote push) and one at the end (no CTA exits while a peer may still push
// into it) are the only cluster-wide barriers.
// ======================================================================
constexpr int kRingCtrl = 2304;
constexpr int kMaxRing = 32;
constexpr int kMaxAffine = 8;  // affine slots (resident mode: chunks per slice)
// Control area layout:
//   [0, 256)       full[32] mbarriers
//   [256, 512)     empty[32] mbarriers
//   [512, 544)     exchange mbarriers [stage][parity]
//   [544, 560)     stats_full[parity] mbarriers
//   [560, 576)     stats_empty[parity] mbarriers
//   [576, 640)     published row statistics [parity][8 floats]
//   [640, 1152)    reduction scratch (128 floats)
//   [1152, 2176)   DSMEM slots [stage][parity][16 sources][4 floats]
//   [2176, 2240)   affine_full[8] mbarriers
//   [2240, 2304)   affine_empty[8] mbarriers
// The chunk ring follows the control area; the affine ring (gamma and beta
// segments of the chunk the writers are on, `affine` slots) follows the ring.

__device__ __forceinline__ float *slot_ptr(float *slots, int stage, int par, int c) {
    return slots + ((stage * 2 + par) * 16 + c) * 4;
}

// All-reduce over the Tc consumer threads (named barrier 1).
template <bool MAX>
__device__ __forceinline__ float cons_allreduce(float v, float *red, int Tc) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = Tc >> 5;
    v = MAX ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[wid] = v;
    named_bar_sync(1, Tc);
    if (wid == 0) {
        float t = lane < nw ? red[lane] : (MAX ? -INFINITY : 0.0f);
        t = MAX ? warp_max(t) : warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    named_bar_sync(1, Tc);
    return red[32];
}

// Deterministic block reduction of a Stream state; returns the CTA partial
// (p0, p1) in the same format as the staged kernel's partials.
// Tc threads take part (the first Tc of the block); bar_id 0 is
// __syncthreads-equivalent for the whole block, 1 is the consumer barrier.
__device__ __forceinline__ void sync_group(int bar_id, int Tc) {
    if (bar_id == 0) __syncthreads();
    else named_bar_sync(bar_id, Tc);
}

template <int OP>
__device__ __forceinline__ float2 block_reduce_stream(Stream<OP> st, float *red, long long n_c, int bar_id = 0,
                                                      int Tc = 0) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (Tc == 0) Tc = blockDim.x;
    const int nw = Tc >> 5;
    if constexpr (OP == OP_RMS) {
        if (bar_id == 0) return make_float2(block_allreduce<false>(st.ss, red), 0.0f);
        return make_float2(cons_allreduce<false>(st.ss, red, Tc), 0.0f);
    } else if constexpr (OP == OP_Q8) {
        if (bar_id == 0) return make_float2(block_allreduce<true>(st.am, red), 0.0f);
        return make_float2(cons_allreduce<true>(st.am, red, Tc), 0.0f);
    } else if constexpr (OP == OP_LN) {
        st.finish();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float nb = __shfl_xor_sync(0xffffffffu, st.n, o);
            const float mb = __shfl_xor_sync(0xffffffffu, st.mu, o);
            const float qb = __shfl_xor_sync(0xffffffffu, st.m2, o);
            if (lane & o) {  // make the merge order independent of which side holds what
                Stream<OP_LN> t;
                t.n = nb; t.mu = mb; t.m2 = qb;
                t.merge3(st.n, st.mu, st.m2);
                st = t;
            } else {
                st.merge3(nb, mb, qb);
            }
        }
        if (lane == 0) {
            red[3 * wid] = st.n;
            red[3 * wid + 1] = st.mu;
            red[3 * wid + 2] = st.m2;
        }
        sync_group(bar_id, Tc);
        if (wid == 0) {  // the warps' states, merged by a shuffle tree in warp 0
            Stream<OP_LN> t;
            if (lane < nw) {
                t.n = red[3 * lane];
                t.mu = red[3 * lane + 1];
                t.m2 = red[3 * lane + 2];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float nb = __shfl_xor_sync(0xffffffffu, t.n, o);
                const float mb = __shfl_xor_sync(0xffffffffu, t.mu, o);
                const float qb = __shfl_xor_sync(0xffffffffu, t.m2, o);
                if (lane & o) {
                    Stream<OP_LN> u;
                    u.n = nb; u.mu = mb; u.m2 = qb;
                    u.merge3(t.n, t.mu, t.m2);
                    t = u;
                } else {
                    t.merge3(nb, mb, qb);
                }
            }
            if (lane == 0) {
                red[96] = t.mu;
                red[97] = t.m2;
            }
        }
        sync_group(bar_id, Tc);
        (void)n_c;
        const float2 r = make_float2(red[96], red[97]);
        sync_group(bar_id, Tc);
        return r;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float m2 = __shfl_xor_sync(0xffffffffu, st.m, o);
            const float s2 = __shfl_xor_sync(0xffffffffu, st.s, o);
            if (lane & o) {
                Stream<OP> t;
                t.m = m2; t.s = s2;
                t.merge(st.m, st.s);
                st = t;
            } else {
                st.merge(m2, s2);
            }
        }
        if (lane == 0) {
            red[2 * wid] = st.m;
            red[2 * wid + 1] = st.s;
        }
        sync_group(bar_id, Tc);
        if (threadIdx.x == 0) {
            Stream<OP> t;
            for (int w = 0; w < nw; ++w) t.merge(red[2 * w], red[2 * w + 1]);
            red[96] = t.m;
            red[97] = t.s;
        }
        sync_group(bar_id, Tc);
        const float2 r = make_float2(red[96], red[97]);
        sync_group(bar_id, Tc);
        return r;
    }
}

// Replicated push all-gather of NQ floats per CTA (consumer threads only).
template <int NQ>
__device__ __forceinline__ const float *exchange_push(float p0, float p1, float *slots, uint64_t *xbar, int stage,
                                                      int par, uint32_t phase, int P, int c, int Tc, unsigned *err) {
    const int tid = threadIdx.x;
    float *mine = slot_ptr(slots, stage, par, c);
    uint64_t *bar = &xbar[stage * 2 + par];
    if (tid < P) {
        if (tid == c) {
            mine[0] = p0;
            if (NQ == 2) mine[1] = p1;
        } else {
            // order this CTA's earlier reads of the slots before the peer's next writes
            fence_release_smem_cluster();
            const uint32_t raddr = mapa_shared(smem_addr(mine), static_cast<uint32_t>(tid));
            const uint32_t rbar = mapa_shared(smem_addr(bar), static_cast<uint32_t>(tid));
            if (NQ == 2) st_async_v2f32(raddr, p0, p1, rbar);
            else st_async_f32(raddr, p0, rbar);
        }
    }
    if (tid == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>((P - 1) * NQ * 4));
    named_bar_sync(1, Tc);
    mbar_wait_bounded_cluster(bar, phase, err);
    return slot_ptr(slots, stage, par, 0);
}

// Visit the gn 16-byte groups of one staged chunk, groups tid, tid + Tc, ...
// U shared-memory loads are issued before any of them is used.
template <int TIN, class F>
__device__ __forceinline__ void visit_chunk(const unsigned char *cb, int gn, int tid, int Tc, float in_sc, F &&fn) {
    constexpr int V = Fmt<TIN>::V;
    constexpr int U = (V == 16) ? 2 : 4;
    int g = tid;
    for (; g + (U - 1) * Tc < gn; g += U * Tc) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = *reinterpret_cast<const uint4 *>(cb + (g + u * Tc) * 16);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float f[V];
            decode_group<TIN>(w[u], f, in_sc);
            fn(g + u * Tc, f);
        }
    }
    for (; g < gn; g += Tc) {
        float f[V];
        decode_group<TIN>(*reinterpret_cast<const uint4 *>(cb + g * 16), f, in_sc);
        fn(g, f);
    }
}

// visit_chunk on the raw 16-byte groups: fn(group index, group).
template <class F>
__device__ __forceinline__ void visit_chunk_raw(const unsigned char *cb, int gn, int tid, int Tc, F &&fn) {
    constexpr int U = 4;
    int g = tid;
    for (; g + (U - 1) * Tc < gn; g += U * Tc) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = *reinterpret_cast<const uint4 *>(cb + (g + u * Tc) * 16);
#pragma unroll
        for (int u = 0; u < U; ++u) fn(g + u * Tc, w[u]);
    }
    for (; g < gn; g += Tc) fn(g, *reinterpret_cast<const uint4 *>(cb + g * 16));
}

// Reuse pass of the norms over one staged chunk with gamma / beta read from
// global memory (L2): for each batch of U groups every gamma / beta load is
// issued before the batch's shared-memory reads and stores, so their latency
// overlaps instead of following each store.
template <int OP, int TIN, int TOUT, class H>
__device__ __forceinline__ void write_chunk_direct(const unsigned char *cb, int gn, int wt, int Tw, float in_sc,
                                                   const float *gamma, const float *beta, long long i0c,
                                                   unsigned char *out_row, bool out_vec, H &&h) {
    constexpr int V = Fmt<TIN>::V, osz = Fmt<TOUT>::size;
    constexpr int U = (V == 4) ? 4 : (V == 8 ? 2 : 1);
    constexpr int NV = V / 4;  // float4 per group
    for (int g0 = wt; g0 < gn; g0 += U * Tw) {
        float4 gv[U][NV], bv[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u * Tw;
            const long long i0 = i0c + static_cast<long long>(g) * V;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                if (g < gn && gamma) gv[u][k] = __ldg(reinterpret_cast<const float4 *>(gamma + i0) + k);
                else gv[u][k] = make_float4(1.0f, 1.0f, 1.0f, 1.0f);
                if (g < gn && beta) bv[u][k] = __ldg(reinterpret_cast<const float4 *>(beta + i0) + k);
                else bv[u][k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u * Tw;
            if (g < gn) w[u] = *reinterpret_cast<const uint4 *>(cb + g * 16);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int g = g0 + u * Tw;
            if (g >= gn) continue;
            float f[V], y[V];
            decode_group<TIN>(w[u], f, in_sc);
            const float *gf = reinterpret_cast<const float *>(&gv[u][0]);
            const float *bf = reinterpret_cast<const float *>(&bv[u][0]);
#pragma unroll
            for (int q = 0; q < V; ++q) y[q] = h(f[q], gf[q], bf[q]);
            const long long i0 = i0c + static_cast<long long>(g) * V;
#pragma unroll
            for (int hv = 0; hv < V; hv += (V < 8 ? V : 8)) {
                constexpr int SV = V < 8 ? V : 8;
                float ys[SV];
#pragma unroll
                for (int q = 0; q < SV; ++q) ys[q] = y[hv + q];
                store_group<TOUT, SV>(out_row + (i0 + hv) * osz, ys, out_vec);
            }
        }
    }
}

// Phase timestamps (global timer, ns) of the first kTraceCtas CTAs, for the
// first trace_rows rows each: [0] row start, [1] stage-1 sweep done (all
// chunks waited), [2] CTA reduction done, [3] exchange done, [4] reuse pass
// done, [5] producer issued the row's last chunk.
constexpr int kTraceCtas = 32;
constexpr int kTraceFields = 8;
__device__ __forceinline__ void trace_stamp(const RowArgs &a, int rr, int field) {
    if (a.trace != nullptr && blockIdx.x < kTraceCtas && rr < a.trace_rows)
        a.trace[(static_cast<size_t>(blockIdx.x) * a.trace_rows + rr) * kTraceFields + field] = global_timer_ns();
}

template <int OP, int TIN, int TOUT>
__global__ void __launch_bounds__(288, 3) k_ring(const RowArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 32;
    uint64_t *xbar = full + 64;
    uint64_t *stats_full = full + 68;
    uint64_t *stats_empty = full + 70;
    float *pub = reinterpret_cast<float *>(smem + 576);
    float *red = reinterpret_cast<float *>(smem + 640);
    float *slots = reinterpret_cast<float *>(smem + 1152);
    uint64_t *affine_full = reinterpret_cast<uint64_t *>(smem + 2176);
    uint64_t *affine_empty = reinterpret_cast<uint64_t *>(smem + 2240);
    unsigned char *ring = smem + kRingCtrl;

    constexpr int isz = Fmt<TIN>::size, V = Fmt<TIN>::V;
    constexpr int SV = V < 8 ? V : 8;  // outputs produced per step of the reuse pass
    constexpr int osz = Fmt<TOUT>::size;
    constexpr bool kFp8Stage = (TOUT == DT_E4M3) && (OP == OP_LN || OP == OP_RMS);

    const int CH = a.chunk_bytes, K = a.ring, gpc = CH / 16;
    // affine ring: per slot, gamma (gpc*V floats) then beta (gpc*V floats)
    const int A = a.affine;
    const bool has_g = a.gamma != nullptr, has_b = (OP == OP_LN) && a.beta != nullptr;
    const int aseg = gpc * V * 4;  // bytes of one gamma or beta segment
    const int aslot = aseg * ((has_g ? 1 : 0) + (has_b ? 1 : 0));
    unsigned char *aring = ring + static_cast<size_t>(K) * CH;
    const int P = static_cast<int>(cluster_nctarank());
    const int c = P > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const long long ncl = gridDim.x / P, cl = blockIdx.x / P;
    const int tid = threadIdx.x;
    const int Tr = a.reducers, Tp = static_cast<int>(blockDim.x) - 32, Tw = Tp - Tr, Ww = Tw >> 5;
    const long long N = a.cols;

    if (tid == 0) {
        for (int k = 0; k < K; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], static_cast<uint32_t>(Ww));
        }
        for (int k = 0; k < 4; ++k) mbar_init(&xbar[k], 1);
        for (int k = 0; k < 2; ++k) {
            mbar_init(&stats_full[k], 1);
            mbar_init(&stats_empty[k], static_cast<uint32_t>(Ww));
        }
        for (int k = 0; k < A; ++k) {
            mbar_init(&affine_full[k], 1);
            mbar_init(&affine_empty[k], static_cast<uint32_t>(Ww));
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (P > 1) cluster_arrive_release();  // start barrier, split
    bool waited_start = false;

    // Geometry of this CTA's slice of `row`.
    struct RowGeo {
        const unsigned char *in_row;
        RowSlice s;
        long long ng;
        int nch;
        float in_sc;
    };
    auto geo = [&](long long row) {
        RowGeo g;
        g.in_row = a.in + row * a.ld_in * isz;
        g.s = make_slice(reinterpret_cast<uintptr_t>(g.in_row), N, isz, P, c);
        g.ng = g.s.g_hi - g.s.g_lo;
        g.nch = static_cast<int>((g.ng * 16 + CH - 1) / CH);
        g.in_sc = (TIN == DT_E4M3) ? a.in_scale[row] : 1.0f;
        return g;
    };
    auto chunk_ptr = [&](const RingPos &rb, int k) -> const unsigned char * {
        return ring + static_cast<size_t>(rb.at(k).slot) * CH;
    };
    auto chunk_groups = [&](const RowGeo &g, int k) -> int {
        const long long r = g.ng - static_cast<long long>(k) * gpc;
        return static_cast<int>(r < gpc ? r : gpc);
    };
    auto edge_x = [&](const RowGeo &g, int e, long long k) -> float {
        const long long i = e == 0 ? k : g.s.h0 + g.s.G * V + k;
        return decode_one<TIN>(g.in_row + i * isz, g.in_sc);
    };

    if (tid >= Tp) {
        // ========================================================== producer
        if (tid == Tp) {
            RingPos rp(K);
            int prr = 0;
            for (long long row = cl; row < a.rows; row += ncl) {
                const RowGeo g = geo(row);
                const long long body = g.ng * 16;
                const unsigned char *src = g.in_row + g.s.h0 * isz + g.s.g_lo * 16;
                for (long long off = 0; off < body; off += CH, rp.next()) {
                    const int slot = rp.slot;
                    if (rp.lap > 0) mbar_wait_bounded(&empty[slot], rp.prev_parity(), a.err);
                    const uint32_t bytes = static_cast<uint32_t>(body - off < CH ? body - off : CH);
                    // (test_extra_tx: bytes no copy delivers, so this phase cannot complete; the host allows it
                    // only for one row of one chunk, where the barrier is never reused)
                    mbar_arrive_expect_tx(&full[slot], bytes + (rp.lap == 0 && slot == 0 ? a.test_extra_tx : 0));
                    bulk_g2s(ring + static_cast<size_t>(slot) * CH, src + off, bytes, &full[slot]);
                }
                trace_stamp(a, prr++, 5);
            }
        } else if (tid == Tp + 1 && A > 0) {
            // gamma / beta segments of every chunk, in the writers' order
            // (resident: the first row's chunks only, one slot each)
            RingPos ap(A);
            for (long long row = cl; row < a.rows && !(a.affine_resident && row > cl); row += ncl) {
                const RowGeo g = geo(row);
                const long long i_base = g.s.h0 + g.s.g_lo * V;
                for (int k = 0; k < g.nch; ++k, ap.next()) {
                    const int slot = ap.slot;
                    if (ap.lap > 0 && !a.affine_resident) mbar_wait_bounded(&affine_empty[slot], ap.prev_parity(), a.err);
                    const uint32_t bytes = static_cast<uint32_t>(chunk_groups(g, k)) * V * 4;
                    const long long e0 = i_base + static_cast<long long>(k) * gpc * V;
                    unsigned char *dst = aring + static_cast<size_t>(slot) * aslot;
                    mbar_arrive_expect_tx(&affine_full[slot], bytes * ((has_g ? 1u : 0u) + (has_b ? 1u : 0u)));
                    if (has_g) bulk_g2s(dst, a.gamma + e0, bytes, &affine_full[slot]);
                    if (has_b) bulk_g2s(dst + (has_g ? aseg : 0), a.beta + e0, bytes, &affine_full[slot]);
                }
            }
        }
        __syncwarp();
    } else if (tid < Tr) {
        // ========================================================== reducers
        RingPos rb(K);  // ring position of the current row's first chunk
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const RowGeo g = geo(row);
            // edge elements spread one per thread (a row has fewer than 16 of each): head element tid,
            // tail element Tr - 1 - tid; -1 where this thread has none
            const long long k_head = (c == 0 && tid < g.s.h0) ? tid : -1;
            const long long k_tail = (c == P - 1 && Tr - 1 - tid < g.s.t0) ? Tr - 1 - tid : -1;
            const int par = rr & 1;
            const uint32_t xphase = static_cast<uint32_t>((rr >> 1) & 1);
            if (tid == 0) trace_stamp(a, rr, 0);

            // ---------- stage 1 (sweeps wait for each chunk as it lands)
            float part0, part1 = 0.0f;
            const long long n_c = slice_count(g.s, V, P, c);
            {
                Stream<OP> acc;
                for (int k = 0; k < g.nch; ++k) {
                    const RingPos pk = rb.at(k);
                    mbar_wait_bounded(&full[pk.slot], pk.parity(), a.err, a.wait_ns ? a.wait_ns : kWaitLimitNs);
                    visit_chunk_raw(chunk_ptr(rb, k), chunk_groups(g, k), tid, Tr,
                                    [&](int, const uint4 &w) { stream_add_group<OP, TIN>(acc, w, g.in_sc); });
                }
                if (k_head >= 0) acc.add1(edge_x(g, 0, k_head));
                if (k_tail >= 0) acc.add1(edge_x(g, 1, k_tail));
                if (tid == 0) trace_stamp(a, rr, 1);
                const float2 part = block_reduce_stream<OP>(acc, red, n_c, 1, Tr);
                part0 = part.x;
                part1 = part.y;
            }
            if (tid == 0) trace_stamp(a, rr, 2);

            // ---------- DSMEM push all-gather (Eq. 5) and fixed-order combine
            Stats st;
            if (P > 1) {
                if (!waited_start) {
                    cluster_wait_acquire();
                    waited_start = true;
                }
                const float *sl = exchange_push<(OP == OP_RMS || OP == OP_Q8) ? 1 : 2>(part0, part1, slots, xbar, 0,
                                                                                        par, xphase, P, c, Tr, a.err);
                st = combine_partials<OP>(sl, 4, P, g.s, V, N, a.eps);
            } else {
                const float p1[2] = {part0, part1};
                st = combine_partials<OP>(p1, 2, 1, g.s, V, N, a.eps);
            }
            if (tid == 0) trace_stamp(a, rr, 3);

            // ---------- stage 2 (FP8 output of the norms): amax |h(x)|
            float qmul = 1.0f;
            if constexpr (kFp8Stage) {
                const long long i_base = g.s.h0 + g.s.g_lo * V;
                const bool g_vec = a.gamma == nullptr || ((reinterpret_cast<uintptr_t>(a.gamma + g.s.h0) & 15u) == 0);
                const bool b_vec = a.beta == nullptr || ((reinterpret_cast<uintptr_t>(a.beta + g.s.h0) & 15u) == 0);
                float am = 0.0f;
                for (int k = 0; k < g.nch; ++k) {
                    const long long kg = static_cast<long long>(k) * gpc;
                    visit_chunk<TIN>(chunk_ptr(rb, k), chunk_groups(g, k), tid, Tr, g.in_sc,
                                     [&](int gi, const float(&f)[V]) {
#pragma unroll
                                         for (int hv = 0; hv < V; hv += SV) {
                                             float gg[SV], bb[SV];
                                             const long long i0 = i_base + (kg + gi) * V + hv;
                                             load_affine<SV>(a.gamma, i0, g_vec, 1.0f, gg);
                                             load_affine<SV>(a.beta, i0, b_vec, 0.0f, bb);
#pragma unroll
                                             for (int q = 0; q < SV; ++q)
                                                 am = fmaxf(am, fabsf(norm_h<OP>(f[hv + q], st, gg[q],
                                                                                 OP == OP_LN ? bb[q] : 0.0f)));
                                         }
                                     });
                }
                for (int e = 0; e < 2; ++e) {
                    const long long k = e == 0 ? k_head : k_tail;
                    if (k < 0) continue;
                    const long long i = e == 0 ? k : g.s.h0 + g.s.G * V + k;
                    const float gg = a.gamma ? a.gamma[i] : 1.0f;
                    const float bb = (OP == OP_LN && a.beta) ? a.beta[i] : 0.0f;
                    am = fmaxf(am, fabsf(norm_h<OP>(edge_x(g, e, k), st, gg, bb)));
                }
                am = cons_allreduce<true>(am, red, Tr);
                if (P > 1) {
                    const float *sl = exchange_push<1>(am, 0.0f, slots, xbar, 1, par, xphase, P, c, Tr, a.err);
                    am = 0.0f;
                    for (int q = 0; q < P; ++q) am = fmaxf(am, sl[q * 4]);
                }
                qmul = am > 0.0f ? 448.0f / am : 1.0f;
                if (c == 0 && tid == 0) a.out_scale[row] = am > 0.0f ? am / 448.0f : 1.0f;
            }
            if constexpr (OP == OP_SOFTMAX && TOUT == DT_E4M3) {
                if (c == 0 && tid == 0) a.out_scale[row] = (1.0f / st.b) * (1.0f / 448.0f);
            }
            if constexpr (OP == OP_LSE) {
                if (c == 0 && tid == 0) reinterpret_cast<float *>(a.out)[row] = st.a + logf(st.b);
            }
            if constexpr (OP == OP_Q8) {
                if (c == 0 && tid == 0) a.out_scale[row] = st.a;
            }

            // ---------- publish the row statistics to the writers
            if (tid == 0) {
                if (rr >= 2) mbar_wait_bounded(&stats_empty[par], static_cast<uint32_t>(((rr >> 1) - 1) & 1), a.err);
                pub[par * 8 + 0] = st.a;
                pub[par * 8 + 1] = st.b;
                pub[par * 8 + 2] = qmul;
                mbar_arrive(&stats_full[par]);
            }
            rb.advance(g.nch);
        }
    } else {
        // ========================================================== writers
        const int wt = tid - Tr;
        RingPos rb(K);                // ring position of the current row's first chunk
        RingPos wb(A > 0 ? A : 1);    // affine ring position of its first chunk
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const RowGeo g = geo(row);
            const int par = rr & 1;
            mbar_wait_bounded(&stats_full[par], static_cast<uint32_t>((rr >> 1) & 1), a.err);
            Stats st;
            st.a = pub[par * 8 + 0];
            st.b = pub[par * 8 + 1];
            const float qmul = pub[par * 8 + 2];
            __syncwarp();
            if ((wt & 31) == 0) mbar_arrive(&stats_empty[par]);

            if constexpr (OP == OP_LSE) {
                for (int k = 0; k < g.nch; ++k) {
                    __syncwarp();
                    if ((wt & 31) == 0) mbar_arrive(&empty[rb.at(k).slot]);
                }
            } else {
                unsigned char *out_row = a.out + row * a.ld_out * osz;
                const long long i_base = g.s.h0 + g.s.g_lo * V;
                constexpr int vec_bytes = (SV * osz) < 16 ? (SV * osz) : 16;
                const bool out_vec = ((reinterpret_cast<uintptr_t>(out_row) + g.s.h0 * osz) % vec_bytes) == 0;
                const bool g_vec = a.gamma == nullptr || ((reinterpret_cast<uintptr_t>(a.gamma + g.s.h0) & 15u) == 0);
                const bool b_vec = a.beta == nullptr || ((reinterpret_cast<uintptr_t>(a.beta + g.s.h0) & 15u) == 0);
                const float inv = (OP == OP_SOFTMAX) ? 1.0f / st.b : 0.0f;
                const float smul = (TOUT == DT_E4M3) ? 448.0f : inv;  // softmax: y (or its code) = exp(x - M) * smul
                const float cL = (OP == OP_SOFTMAX) ? log2f(smul) : 0.0f;  // exp_sub's log2-domain scale
                auto h = [&](float x, float gm, float bt) -> float {
                    if constexpr (OP == OP_SOFTMAX) return exp_sub(x, st.a, cL);
                    else if constexpr (OP == OP_Q8) return q8_code(x, st.a, st.b);
                    else return norm_h<OP>(x, st, gm, bt) * qmul;
                };
                for (int k = 0; k < g.nch; ++k) {
                    const long long kg = static_cast<long long>(k) * gpc;
                    const int aslot_k = A > 0 ? (a.affine_resident ? k : wb.at(k).slot) : 0;
                    const float *ag = reinterpret_cast<const float *>(aring + static_cast<size_t>(aslot_k) * aslot);
                    const float *ab = ag + (has_g ? gpc * V : 0);
                    if (A > 0 && (!a.affine_resident || rr == 0))
                        mbar_wait_bounded(&affine_full[aslot_k],
                                          a.affine_resident ? 0u : wb.at(k).parity(), a.err);
                    if constexpr (OP == OP_LN || OP == OP_RMS) {
                        if (A == 0 && g_vec && b_vec && (has_g || has_b)) {
                            write_chunk_direct<OP, TIN, TOUT>(chunk_ptr(rb, k), chunk_groups(g, k), wt, Tw, g.in_sc,
                                                              has_g ? a.gamma : nullptr, has_b ? a.beta : nullptr,
                                                              i_base + kg * V, out_row, out_vec, h);
                            __syncwarp();
                            if ((wt & 31) == 0) mbar_arrive(&empty[rb.at(k).slot]);
                            continue;
                        }
                    }
                    if constexpr (OP == OP_SOFTMAX && TIN == DT_E4M3 && TOUT == DT_E4M3) {
                        // raw codes in and out (softmax_e4m3_codes), 16-byte stores: only where the output
                        // groups start on the 16-byte grid (out_vec checks 8 bytes for this format)
                        if (((reinterpret_cast<uintptr_t>(out_row) + g.s.h0) & 15u) == 0) {
                            const uint32_t neg = e4m3_sign_mask(g.in_sc);
                            const float a1 = fabsf(g.in_sc);
                            visit_chunk_raw(chunk_ptr(rb, k), chunk_groups(g, k), wt, Tw, [&](int gi, const uint4 &w) {
                                *reinterpret_cast<uint4 *>(out_row + i_base + (kg + gi) * V) =
                                    softmax_e4m3_codes(e4m3_fold_sign(w, neg), a1, st.a);
                            });
                            __syncwarp();
                            if ((wt & 31) == 0) mbar_arrive(&empty[rb.at(k).slot]);
                            continue;
                        }
                    }
                    visit_chunk<TIN>(chunk_ptr(rb, k), chunk_groups(g, k), wt, Tw, g.in_sc,
                                     [&](int gi, const float(&f)[V]) {
#pragma unroll
                                         for (int hv = 0; hv < V; hv += SV) {
                                             float gg[SV], bb[SV], y[SV];
                                             const long long i0 = i_base + (kg + gi) * V + hv;
                                             if constexpr (OP == OP_LN || OP == OP_RMS) {
                                                 if (A > 0) load_affine_smem<SV>(has_g ? ag : nullptr, gi * V + hv, 1.0f, gg);
                                                 else load_affine<SV>(a.gamma, i0, g_vec, 1.0f, gg);
                                             }
                                             if constexpr (OP == OP_LN) {
                                                 if (A > 0) load_affine_smem<SV>(has_b ? ab : nullptr, gi * V + hv, 0.0f, bb);
                                                 else load_affine<SV>(a.beta, i0, b_vec, 0.0f, bb);
                                             }
#pragma unroll
                                             for (int q = 0; q < SV; ++q)
                                                 y[q] = h(f[hv + q], (OP == OP_LN || OP == OP_RMS) ? gg[q] : 1.0f,
                                                          OP == OP_LN ? bb[q] : 0.0f);
                                             store_group<TOUT, SV>(out_row + i0 * osz, y, out_vec);
                                         }
                                     });
                    __syncwarp();
                    if ((wt & 31) == 0) {
                        mbar_arrive(&empty[rb.at(k).slot]);
                        if (A > 0 && !a.affine_resident) mbar_arrive(&affine_empty[aslot_k]);
                    }
                }
                wb.advance(g.nch);
                // edge elements, one per writer thread (head element wt, tail element Tw - 1 - wt)
                for (int e = 0; e < 2; ++e) {
                    const long long k = e == 0 ? ((c == 0 && wt < g.s.h0) ? wt : -1)
                                               : ((c == P - 1 && Tw - 1 - wt < g.s.t0) ? Tw - 1 - wt : -1);
                    if (k < 0) continue;
                    const long long i = e == 0 ? k : g.s.h0 + g.s.G * V + k;
                    const float gm = ((OP == OP_LN || OP == OP_RMS) && a.gamma) ? a.gamma[i] : 1.0f;
                    const float bt = (OP == OP_LN && a.beta) ? a.beta[i] : 0.0f;
                    store_one<TOUT>(out_row + i * osz, h(edge_x(g, e, k), gm, bt));
                }
            }
            if (wt == 0) trace_stamp(a, rr, 4);
            rb.advance(g.nch);
        }
    }
    if (P > 1) {
        if (!waited_start) cluster_wait_acquire();
        cluster_arrive_release();  // end barrier: nobody exits while a peer may push into it
        cluster_wait_acquire();
    }
}

// Visit this CTA's part of a row in global memory, 4 groups in flight per thread.
// L2 treatment of a sweep's loads: 0 default, 1 keep (the row is read again
// soon), 2 evict first (last read).
template <int L2H>
__device__ __forceinline__ uint64_t sweep_policy() {
    if constexpr (L2H == 1) return l2_evict_last_policy();
    else if constexpr (L2H == 2) return l2_evict_first_policy();
    else return 0;
}
template <int L2H>
__device__ __forceinline__ uint4 sweep_load(const unsigned char *p, uint64_t pol) {
    if constexpr (L2H == 0) return ld_global_v4(p);
    else return ld_global_v4_hint(p, pol);
}

template <int TIN, int L2H = 0, class F>
__device__ __forceinline__ void sweep_global(const unsigned char *in_row, const RowSlice &s, int P, int c,
                                             float in_sc, F &&fn /* fn(long long elem_index, float(&)[V]) */) {
    constexpr int V = Fmt<TIN>::V, isz = Fmt<TIN>::size;
    const int tid = threadIdx.x, T = blockDim.x;
    const unsigned char *body = in_row + s.h0 * isz;
    const uint64_t pol = sweep_policy<L2H>();
    constexpr int U = 4;  // 16-byte loads in flight per thread (8 spills at 64 registers and measures slower)
    for (long long g0 = s.g_lo + tid; g0 < s.g_hi; g0 += static_cast<long long>(U) * T) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + static_cast<long long>(u) * T;
            if (g < s.g_hi) w[u] = sweep_load<L2H>(body + g * 16, pol);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + static_cast<long long>(u) * T;
            if (g < s.g_hi) {
                float f[V];
                decode_group<TIN>(w[u], f, in_sc);
                fn(s.h0 + g * V, f);
            }
        }
    }
    (void)P;
    (void)c;
}

// sweep_global on the raw 16-byte groups: fn(first element index, group).
template <int TIN, int L2H = 0, class F>
__device__ __forceinline__ void sweep_global_raw(const unsigned char *in_row, const RowSlice &s,
                                                 F &&fn /* fn(long long elem_index, const uint4 &) */) {
    constexpr int V = Fmt<TIN>::V, isz = Fmt<TIN>::size;
    const int tid = threadIdx.x, T = blockDim.x;
    const unsigned char *body = in_row + s.h0 * isz;
    const uint64_t pol = sweep_policy<L2H>();
    constexpr int U = 4;
    for (long long g0 = s.g_lo + tid; g0 < s.g_hi; g0 += static_cast<long long>(U) * T) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + static_cast<long long>(u) * T;
            if (g < s.g_hi) w[u] = sweep_load<L2H>(body + g * 16, pol);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long g = g0 + static_cast<long long>(u) * T;
            if (g < s.g_hi) fn(s.h0 + g * V, w[u]);
        }
    }
}

// Edge elements of this CTA, one per thread (a row has fewer than 16 head and
// 16 tail elements): head element t by thread t of CTA 0, tail element k by
// thread T - 1 - k of CTA P-1, so their loads are in flight together.
template <int TIN, class F>
__device__ __forceinline__ void sweep_edges(const unsigned char *in_row, const RowSlice &s, int P, int c, float in_sc,
                                            F &&fn /* fn(long long i, float x) */) {
    constexpr int V = Fmt<TIN>::V, isz = Fmt<TIN>::size;
    const long long t = threadIdx.x, kt = static_cast<long long>(blockDim.x) - 1 - t;
    if (c == 0 && t < s.h0) fn(t, decode_one<TIN>(in_row + t * isz, in_sc));
    if (c == P - 1 && kt < s.t0) {
        const long long i = s.h0 + s.G * V + kt;
        fn(i, decode_one<TIN>(in_row + i * isz, in_sc));
    }
}

template <int OP, int TIN, int L2H = 0>
__device__ __forceinline__ float2 stats_sweep(const RowArgs &a, const unsigned char *in_row, const RowSlice &s, int P,
                                              int c, float in_sc, float *red) {
    Stream<OP> st;
    sweep_global_raw<TIN, L2H>(in_row, s, [&](long long, const uint4 &w) { stream_add_group<OP, TIN>(st, w, in_sc); });
    sweep_edges<TIN>(in_row, s, P, c, in_sc, [&](long long, float x) { st.add1(x); });
    return block_reduce_stream<OP>(st, red, slice_count(s, Fmt<TIN>::V, P, c));
}

template <int OP, int TIN, int L2H = 0>
__device__ __forceinline__ float amax_sweep(const RowArgs &a, const unsigned char *in_row, const RowSlice &s, int P,
                                            int c, float in_sc, const Stats &st, float *red) {
    constexpr int V = Fmt<TIN>::V;
    const bool g_vec = a.gamma == nullptr || ((reinterpret_cast<uintptr_t>(a.gamma + s.h0) & 15u) == 0);
    const bool b_vec = a.beta == nullptr || ((reinterpret_cast<uintptr_t>(a.beta + s.h0) & 15u) == 0);
    float am = 0.0f;
    sweep_global<TIN, L2H>(in_row, s, P, c, in_sc, [&](long long i0, const float(&f)[V]) {
        float gg[V], bb[V];
        load_affine<V>(a.gamma, i0, g_vec, 1.0f, gg);
        load_affine<V>(a.beta, i0, b_vec, 0.0f, bb);
#pragma unroll
        for (int j = 0; j < V; ++j) am = fmaxf(am, fabsf(norm_h<OP>(f[j], st, gg[j], OP == OP_LN ? bb[j] : 0.0f)));
    });
    sweep_edges<TIN>(in_row, s, P, c, in_sc, [&](long long i, float x) {
        const float gg = a.gamma ? a.gamma[i] : 1.0f, bb = (OP == OP_LN && a.beta) ? a.beta[i] : 0.0f;
        am = fmaxf(am, fabsf(norm_h<OP>(x, st, gg, bb)));
    });
    return block_allreduce<true>(am, red);
}

template <int OP, int TIN, int TOUT, int L2H = 0>
__device__ __forceinline__ void apply_sweep(const RowArgs &a, long long row, const unsigned char *in_row,
                                            const RowSlice &s, int P, int c, float in_sc, const Stats &st,
                                            float qmul) {
    constexpr int V = Fmt<TIN>::V, osz = Fmt<TOUT>::size;
    unsigned char *out_row = a.out + row * a.ld_out * osz;
    constexpr int vec_bytes = (V * osz) < 16 ? (V * osz) : 16;
    const bool out_vec = ((reinterpret_cast<uintptr_t>(out_row) + s.h0 * osz) % vec_bytes) == 0;
    const bool g_vec = a.gamma == nullptr || ((reinterpret_cast<uintptr_t>(a.gamma + s.h0) & 15u) == 0);
    const bool b_vec = a.beta == nullptr || ((reinterpret_cast<uintptr_t>(a.beta + s.h0) & 15u) == 0);
    if constexpr (OP == OP_SOFTMAX && TIN == DT_E4M3 && TOUT == DT_E4M3) {
        // E4M3 codes in and out, from the raw input codes (softmax_e4m3_codes)
        const float M = st.a, a1 = fabsf(in_sc), c8 = log2f(448.0f);
        const uint32_t neg = e4m3_sign_mask(in_sc);
        sweep_global_raw<TIN, L2H>(in_row, s, [&](long long i0, const uint4 &w0) {
            const uint4 o = softmax_e4m3_codes(e4m3_fold_sign(w0, neg), a1, M);
            unsigned char *p = out_row + i0;
            if (out_vec) {
                if constexpr (L2H == 0) *reinterpret_cast<uint4 *>(p) = o;
                else st_global_v4_hint(p, o, l2_evict_first_policy());
            } else {
                const uint32_t ow[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                for (int k = 0; k < 16; ++k) p[k] = static_cast<unsigned char>(ow[k >> 2] >> (8 * (k & 3)));
            }
        });
        sweep_edges<TIN>(in_row, s, P, c, in_sc,
                         [&](long long i, float x) { store_one<TOUT>(out_row + i, exp_sub(x, M, c8)); });
    } else if constexpr (OP == OP_SOFTMAX) {
        // y (or its FP8 code) = exp(x - M) * mul = 2^((x - M) log2 e + log2 mul)
        const float mul = (TOUT == DT_E4M3) ? 448.0f : 1.0f / st.b;
        const float cL = log2f(mul);
        sweep_global<TIN, L2H>(in_row, s, P, c, in_sc, [&](long long i0, const float(&f)[V]) {
            float y[V];
            exp_sub_group<V>(f, st.a, cL, y);
            store_group<TOUT, V>(out_row + i0 * osz, y, out_vec);
        });
        sweep_edges<TIN>(in_row, s, P, c, in_sc,
                         [&](long long i, float x) { store_one<TOUT>(out_row + i * osz, exp_sub(x, st.a, cL)); });
    } else if constexpr (OP == OP_Q8) {
        sweep_global<TIN, L2H>(in_row, s, P, c, in_sc, [&](long long i0, const float(&f)[V]) {
            float y[V];
            q8_codes<V>(f, st.a, st.b, y);
            store_group<TOUT, V>(out_row + i0 * osz, y, out_vec);
        });
        sweep_edges<TIN>(in_row, s, P, c, in_sc,
                         [&](long long i, float x) { store_one<TOUT>(out_row + i * osz, q8_code(x, st.a, st.b)); });
    } else {
        sweep_global<TIN, L2H>(in_row, s, P, c, in_sc, [&](long long i0, const float(&f)[V]) {
            float gg[V], bb[V], y[V];
            load_affine<V>(a.gamma, i0, g_vec, 1.0f, gg);
            if constexpr (OP == OP_LN) load_affine<V>(a.beta, i0, b_vec, 0.0f, bb);
#pragma unroll
            for (int j = 0; j < V; ++j) y[j] = norm_h<OP>(f[j], st, gg[j], OP == OP_LN ? bb[j] : 0.0f) * qmul;
            store_group<TOUT, V>(out_row + i0 * osz, y, out_vec);
        });
        sweep_edges<TIN>(in_row, s, P, c, in_sc, [&](long long i, float x) {
            const float gg = a.gamma ? a.gamma[i] : 1.0f, bb = (OP == OP_LN && a.beta) ? a.beta[i] : 0.0f;
            store_one<TOUT>(out_row + i * osz, norm_h<OP>(x, st, gg, bb) * qmul);
        });
    }
}

// ----------------------------------------------------------------------
// E4M3 softmax / log-sum-exp rows through per-row code tables (one CTA per
// row).  A row of E4M3 codes b with scale a takes at most 256 values
// x(b) = a value(b), so a statistics term exp(x - m) for a fixed m, and an
// FP8 softmax output code, depend on the input code alone: the CTA evaluates
// them once per code into a shared-memory table, and every element costs one
// table lookup instead of a decode, an FMA chain and an SFU exponential.
// The table keeps 32 copies of each entry, (b, lane) at b * 32 + lane, so the
// 32 lookups of a warp hit 32 different banks whatever the codes are.
// ----------------------------------------------------------------------
constexpr int kLutLanes = 32;
constexpr int kLutEntries = 256 * kLutLanes;
// The terms are first taken about m0 = |a| 448, which bounds every finite x
// of the row.  Their sum S0 = sum exp(x - m0) is kept when S0 >= 2^-8: then
// each term that matters has |x - m0| < (8 + log2 cols) ln 2, so the relative
// error of a term (from rounding x - m0 and the exponent) stays a few 1e-7
// times that, a few 1e-6 at most.  A row whose largest value lies further
// below m0 is summed again about its own maximum.
constexpr float kLutMinSum = 0.00390625f;  // 2^-8

__device__ __forceinline__ float e4m3_value(uint32_t b) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(b & 0xFFu), __NV_E4M3)));
}

// Fill a table: the 32 copies of entry b = val(b).  Warp w evaluates the codes
// 32 k + lane of the blocks k = w, w + warps, ...; each value then goes to its
// 32 copies by a shuffle and 16-byte stores (8 lanes per entry).
template <class F>
__device__ __forceinline__ void lut_fill(uint32_t *tab, F &&val) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int blk = threadIdx.x >> 5; blk < 8; blk += nw) {
        const uint32_t mine = val(static_cast<uint32_t>(blk * 32 + lane));
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int r = 4 * k + (lane >> 3);
            const uint32_t v = __shfl_sync(0xffffffffu, mine, r);
            reinterpret_cast<uint4 *>(tab + (blk * 32 + r) * kLutLanes)[lane & 7] = make_uint4(v, v, v, v);
        }
    }
}

// Maximum of 16 sign-folded E4M3 codes, on FP16 halves (E4M3 is a subset of FP16).
__device__ __forceinline__ __half2 e4m3_group_hmax(const uint4 &w) {
    __half2 h[8];
    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        __half2_raw r0 = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(u[k] & 0xFFFFu), __NV_E4M3);
        __half2_raw r1 = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(u[k] >> 16), __NV_E4M3);
        h[2 * k] = *reinterpret_cast<__half2 *>(&r0);
        h[2 * k + 1] = *reinterpret_cast<__half2 *>(&r1);
    }
    return __hmax2(__hmax2(__hmax2(h[0], h[1]), __hmax2(h[2], h[3])), __hmax2(__hmax2(h[4], h[5]), __hmax2(h[6], h[7])));
}

// Entry of code byte I of u in this lane's copy of a table (base: the table's shared-memory address + 4 lane):
// the byte moved down by one permute, the address by one shift-add, one 32-bit shared load.
template <int I>
__device__ __forceinline__ uint32_t lut_ld(uint32_t base, uint32_t u) {
    const uint32_t b = __byte_perm(u, 0u, 0x4440u | I);
    uint32_t v;
    asm("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(base + (b << 7)));
    return v;
}
__device__ __forceinline__ uint32_t lut_base(const uint32_t *tab) { return smem_addr(tab) + 4u * (threadIdx.x & 31); }

// Sum of the table entries of this thread's codes (16 lookups per group, summed as a tree); with MAXT also
// their running maximum (the entries increase with x).
template <bool MAXT, int L2H>
__device__ __forceinline__ float lut_sum_sweep(const unsigned char *in_row, const RowSlice &s, const uint32_t *tab,
                                               float &tmax) {
    const uint32_t base = lut_base(tab);
    float sum = 0.0f;
    sweep_global_raw<DT_E4M3, L2H>(in_row, s, [&](long long, const uint4 &w) {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
        float e[16];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            e[4 * k] = __uint_as_float(lut_ld<0>(base, u[k]));
            e[4 * k + 1] = __uint_as_float(lut_ld<1>(base, u[k]));
            e[4 * k + 2] = __uint_as_float(lut_ld<2>(base, u[k]));
            e[4 * k + 3] = __uint_as_float(lut_ld<3>(base, u[k]));
        }
        sum += sum_tree<16>(e);
        if constexpr (MAXT) tmax = fmaxf(tmax, max_of(e));
    });
    return sum;
}

// The statistics table about m: entry b = 2^((a value(b) - m) log2 e), flushed below 2^-126 (a flushed
// term is < 2^-126 m-relative, as in the online form), the difference rounded once.
__device__ __forceinline__ void lut_fill_terms(uint32_t *tab, float in_sc, float m) {
    lut_fill(tab, [&](uint32_t b) { return __float_as_uint(ex2_ftz(fmaf(e4m3_value(b), in_sc, -m) * kLog2e)); });
}

// sum exp(x - m) over the row: table about m, one sweep, the edge elements directly, block sum.
template <int L2H>
__device__ __forceinline__ float lut_row_sum(const unsigned char *in_row, const RowSlice &s, float in_sc, float m,
                                             uint32_t *tab, float *red) {
    __syncthreads();  // the previous table's lookups are done
    lut_fill_terms(tab, in_sc, m);
    __syncthreads();
    float tmax = 0.0f;
    float sum = lut_sum_sweep<false, L2H>(in_row, s, tab, tmax);
    sweep_edges<DT_E4M3>(in_row, s, 1, 0, in_sc, [&](long long, float x) { sum += ex2_ftz((x - m) * kLog2e); });
    return block_allreduce<false>(sum, red);
}

// The row maximum of x: the sign-folded codes' maximum on FP16 halves, scaled, and the edge elements'
// maximum xm of this thread.
__device__ __forceinline__ float lut_row_max(const unsigned char *in_row, const RowSlice &s, float in_sc, float xm,
                                             float *red) {
    const uint32_t neg = e4m3_sign_mask(in_sc);
    __half2 hm = __half2half2(__ushort_as_half(0xFC00u));  // -inf
    sweep_global_raw<DT_E4M3, 1>(in_row, s, [&](long long, const uint4 &w) {
        hm = __hmax2(hm, e4m3_group_hmax(e4m3_fold_sign(w, neg)));
    });
    const float q = fmaxf(__low2float(hm), __high2float(hm));
    return block_allreduce<true>(fmaxf(q == -INFINITY ? -INFINITY : q * fabsf(in_sc), xm), red);
}

template <int OP, int TOUT>
__device__ __forceinline__ void tp_fused_e4m3(const RowArgs &a, long long row, const unsigned char *in_row,
                                              const RowSlice &s, float in_sc, float *red) {
    __shared__ __align__(16) uint32_t tab[kLutEntries];
    const float m0 = fabsf(in_sc) * 448.0f;
    // sweep 1: terms about m0 (and, for softmax, their maximum); the row is kept in L2 for the next sweep
    lut_fill_terms(tab, in_sc, m0);
    __syncthreads();
    float tmax = 0.0f;
    float sum = lut_sum_sweep<OP == OP_SOFTMAX, OP == OP_SOFTMAX ? 1 : 0>(in_row, s, tab, tmax);
    float xm = -INFINITY;
    sweep_edges<DT_E4M3>(in_row, s, 1, 0, in_sc, [&](long long, float x) {
        sum += ex2_ftz((x - m0) * kLog2e);
        xm = fmaxf(xm, x);
    });
    const float S0 = block_allreduce<false>(sum, red);
    if constexpr (OP == OP_LSE) {
        float lse = m0 + logf(S0);
        if (!(S0 >= kLutMinSum)) {
            // the row's maximum lies far below m0: find it, then sum about it
            const float M = lut_row_max(in_row, s, in_sc, xm, red);
            lse = M + logf(lut_row_sum<0>(in_row, s, in_sc, M, tab, red));
        }
        if (threadIdx.x == 0) reinterpret_cast<float *>(a.out)[row] = lse;
    } else {
        float M, S;
        if (S0 >= kLutMinSum) {
            // the row maximum from the largest entry met: the largest value among the codes with that entry
            // (a code not in the row can share it only if its value is within ~1e-6 of the maximum)
            const float Tm = block_allreduce<true>(tmax, red);
            float cand = xm;
            for (int b = threadIdx.x; b < 256; b += blockDim.x)
                if (__uint_as_float(tab[b * kLutLanes]) == Tm) cand = fmaxf(cand, e4m3_value(b) * in_sc);
            M = block_allreduce<true>(cand, red);
            S = M == m0 ? S0 : S0 * ex2_ftz((m0 - M) * kLog2e);
        } else {
            M = lut_row_max(in_row, s, in_sc, xm, red);
            S = lut_row_sum<1>(in_row, s, in_sc, M, tab, red);
        }
        if constexpr (TOUT == DT_E4M3) {
            if (threadIdx.x == 0) a.out_scale[row] = (1.0f / S) * (1.0f / 448.0f);
            // sweep 2: output code of input code b = E4M3(448 exp(x(b) - M)), evaluated once per code in FP32
            const float c8 = log2f(448.0f);
            __syncthreads();  // the statistics table's last reads (the maximum's codes) are done
            lut_fill(tab, [&](uint32_t b) {
                const float d = fmaf(e4m3_value(b), in_sc, -M);
                return static_cast<uint32_t>(__nv_cvt_float_to_fp8(ex2_ftz(fmaf(d, kLog2e, c8 + kExpLift)) * kExpDrop,
                                                                   __NV_SATFINITE, __NV_E4M3));
            });
            __syncthreads();
            unsigned char *out_row = a.out + row * a.ld_out;
            const bool out_vec = ((reinterpret_cast<uintptr_t>(out_row) + s.h0) & 15u) == 0;
            const uint32_t base = lut_base(tab);
            const uint64_t pol = l2_evict_first_policy();
            // one sweep per store form, so the loop body holds only the stores it executes
            auto sweep = [&](auto vec) {
                sweep_global_raw<DT_E4M3, 2>(in_row, s, [&](long long i0, const uint4 &w) {
                    const uint32_t u[4] = {w.x, w.y, w.z, w.w};
                    uint32_t o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        o[k] = __byte_perm(__byte_perm(lut_ld<0>(base, u[k]), lut_ld<1>(base, u[k]), 0x0040),
                                           __byte_perm(lut_ld<2>(base, u[k]), lut_ld<3>(base, u[k]), 0x0040), 0x5410);
                    unsigned char *p = out_row + i0;
                    if constexpr (decltype(vec)::value) {
                        st_global_v4_hint(p, make_uint4(o[0], o[1], o[2], o[3]), pol);
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k) p[k] = static_cast<unsigned char>(o[k >> 2] >> (8 * (k & 3)));
                    }
                });
            };
            if (out_vec) sweep(std::true_type{});
            else sweep(std::false_type{});
            sweep_edges<DT_E4M3>(in_row, s, 1, 0, in_sc,
                                 [&](long long i, float x) { store_one<DT_E4M3>(out_row + i, exp_sub(x, M, c8)); });
        } else {
            const Stats st{M, S};
            apply_sweep<OP, DT_E4M3, TOUT, 2>(a, row, in_row, s, 1, 0, in_sc, st, 1.0f);
        }
    }
}

// ----------------------------------------------------------------------
// Two-pass path, one CTA per row (single launch, the row is read twice).
// ----------------------------------------------------------------------
template <int OP, int TIN, int TOUT>
__global__ void __launch_bounds__(1024) k_tp_fused(const RowArgs a) {
    __shared__ float red[128];
    constexpr int isz = Fmt<TIN>::size, V = Fmt<TIN>::V;
    const long long row = blockIdx.x + a.row0;
    const unsigned char *in_row = a.in + row * a.ld_in * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(in_row), a.cols, isz, 1, 0);
    const float in_sc = (TIN == DT_E4M3) ? a.in_scale[row] : 1.0f;
    if constexpr (TIN == DT_E4M3 && (OP == OP_SOFTMAX || OP == OP_LSE)) {
        tp_fused_e4m3<OP, TOUT>(a, row, in_row, s, in_sc, red);
        return;
    }
    // the row is read again by this CTA right after (not for log-sum-exp): its lines are kept in L2 on the
    // first read and go first on the second
    const float2 p = stats_sweep<OP, TIN, OP == OP_LSE ? 0 : 1>(a, in_row, s, 1, 0, in_sc, red);
    const float pp[2] = {p.x, p.y};
    const Stats st = combine_partials<OP>(pp, 2, 1, s, V, a.cols, a.eps);
    if constexpr (OP == OP_LSE) {
        if (threadIdx.x == 0) reinterpret_cast<float *>(a.out)[row] = st.a + logf(st.b);
    } else {
        float qmul = 1.0f;
        if constexpr (TOUT == DT_E4M3 && (OP == OP_LN || OP == OP_RMS)) {
            const float am = amax_sweep<OP, TIN, 1>(a, in_row, s, 1, 0, in_sc, st, red);
            qmul = am > 0.0f ? 448.0f / am : 1.0f;
            if (threadIdx.x == 0) a.out_scale[row] = am > 0.0f ? am / 448.0f : 1.0f;
        }
        if constexpr (TOUT == DT_E4M3 && OP == OP_SOFTMAX) {
            if (threadIdx.x == 0) a.out_scale[row] = (1.0f / st.b) * (1.0f / 448.0f);
        }
        if constexpr (OP == OP_Q8) {
            if (threadIdx.x == 0) a.out_scale[row] = st.a;
        }
        apply_sweep<OP, TIN, TOUT, 2>(a, row, in_row, s, 1, 0, in_sc, st, qmul);
    }
}

// ----------------------------------------------------------------------
// Two-pass path, G CTAs per row (workspace partials, launches as barriers).
// Grid: G * rows_in_launch; CTA (r, g) = blockIdx.x / G, blockIdx.x % G.
// ws layout: [(row - row0) * G + g] * 4 floats: stats partial in [0, 2),
// amax partial in [2].
// ----------------------------------------------------------------------
template <int OP, int TIN>
__global__ void __launch_bounds__(1024) k_tp_stats(const RowArgs a) {
    __shared__ float red[128];
    constexpr int isz = Fmt<TIN>::size;
    const int G = a.G, g = blockIdx.x % G;
    const long long lr = blockIdx.x / G, row = lr + a.row0;
    const unsigned char *in_row = a.in + row * a.ld_in * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(in_row), a.cols, isz, G, g);
    const float in_sc = (TIN == DT_E4M3) ? a.in_scale[row] : 1.0f;
    const float2 p = stats_sweep<OP, TIN>(a, in_row, s, G, g, in_sc, red);
    if (threadIdx.x == 0) {
        float *w = a.ws + (lr * G + g) * 4;
        w[0] = p.x;
        w[1] = p.y;
    }
}

template <int OP, int TIN>
__device__ __forceinline__ Stats tp_row_stats(const RowArgs &a, long long lr, const RowSlice &s) {
    return combine_partials<OP>(a.ws + lr * a.G * 4, 4, a.G, s, Fmt<TIN>::V, a.cols, a.eps);
}

template <int OP, int TIN>
__global__ void __launch_bounds__(1024) k_tp_amax(const RowArgs a) {
    __shared__ float red[128];
    constexpr int isz = Fmt<TIN>::size;
    const int G = a.G, g = blockIdx.x % G;
    const long long lr = blockIdx.x / G, row = lr + a.row0;
    const unsigned char *in_row = a.in + row * a.ld_in * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(in_row), a.cols, isz, G, g);
    const float in_sc = (TIN == DT_E4M3) ? a.in_scale[row] : 1.0f;
    const Stats st = tp_row_stats<OP, TIN>(a, lr, s);
    const float am = amax_sweep<OP, TIN>(a, in_row, s, G, g, in_sc, st, red);
    if (threadIdx.x == 0) a.ws[(lr * G + g) * 4 + 2] = am;
}

template <int OP, int TIN, int TOUT>
__global__ void __launch_bounds__(1024) k_tp_apply(const RowArgs a) {
    constexpr int isz = Fmt<TIN>::size;
    const int G = a.G, g = blockIdx.x % G;
    const long long lr = blockIdx.x / G, row = lr + a.row0;
    const unsigned char *in_row = a.in + row * a.ld_in * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(in_row), a.cols, isz, G, g);
    const float in_sc = (TIN == DT_E4M3) ? a.in_scale[row] : 1.0f;
    const Stats st = tp_row_stats<OP, TIN>(a, lr, s);
    float qmul = 1.0f;
    if constexpr (TOUT == DT_E4M3 && (OP == OP_LN || OP == OP_RMS)) {
        float am = 0.0f;
        for (int k = 0; k < G; ++k) am = fmaxf(am, a.ws[(lr * G + k) * 4 + 2]);
        qmul = am > 0.0f ? 448.0f / am : 1.0f;
        if (g == 0 && threadIdx.x == 0) a.out_scale[row] = am > 0.0f ? am / 448.0f : 1.0f;
    }
    if constexpr (TOUT == DT_E4M3 && OP == OP_SOFTMAX) {
        if (g == 0 && threadIdx.x == 0) a.out_scale[row] = (1.0f / st.b) * (1.0f / 448.0f);
    }
    if constexpr (OP == OP_Q8) {
        if (g == 0 && threadIdx.x == 0) a.out_scale[row] = st.a;
    }
    apply_sweep<OP, TIN, TOUT>(a, row, in_row, s, G, g, in_sc, st, qmul);
}

// One thread per row: combine the G log-sum-exp partials.
template <int TIN>
__global__ void k_tp_lse_final(const RowArgs a, long long nrows) {
    const long long lr = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (lr >= nrows) return;
    const long long row = lr + a.row0;
    const RowSlice s = make_slice(0, a.cols, Fmt<TIN>::size, a.G, 0);
    const Stats st = combine_partials<OP_LSE>(a.ws + lr * a.G * 4, 4, a.G, s, Fmt<TIN>::V, a.cols, a.eps);
    reinterpret_cast<float *>(a.out)[row] = st.a + logf(st.b);
}

// ----------------------------------------------------------------------
// Kernel table of one (input dtype) translation unit.
// ----------------------------------------------------------------------
struct KernelSet {
    const void *ring;
    const void *ring_tm;  // TMEM retention variant (null where it does not apply)
    const void *tp_fused;
    const void *tp_stats;
    const void *tp_amax;
    const void *tp_apply;
    const void *tp_lse_final;
};

}  // namespace credit
