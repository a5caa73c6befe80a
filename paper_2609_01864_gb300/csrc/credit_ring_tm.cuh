// credit_ring_tm.cuh -- the staged path with tensor memory as the retention tier.
//
// Same method as k_ring (Eq. 2 slicing, one sweep that reduces a slice while
// it lands, Eq. 5 push exchange, a combine in one fixed order in every CTA,
// reuse pass from on-chip storage), with the retained slice held in tensor
// memory (TMEM: 128 lanes x 512 32-bit columns = 256 KiB per SM) instead of
// the shared-memory ring:
//
//   producer (warp 16, lane 0)  streams the slice's chunks into a short
//            shared-memory ring with cp.async.bulk, as in k_ring; lane 1
//            stages gamma / beta (resident, or streamed chunk by chunk).
//   reducers (warps 0-7)  take each chunk as it lands.  TMEM lane t (of 128)
//            holds groups t, t + 128, ... of every chunk; reducer thread
//            r owns lane r % 128 and half r / 128 of the lane's kTmGroups
//            groups.  Each thread loads its groups into registers, releases
//            the ring slot at once, adds them to its running statistics and
//            stores the raw bytes into its lane (tcgen05.st).  At the end of
//            the slice each warp merges its lanes (shuffle tree) and pushes
//            the warp's partial into its slot in every CTA of the cluster,
//            its own included (st.async, Eq. 5, one partial per warp instead
//            of one per CTA), and goes straight on to the next row: no
//            CTA-wide barrier, no wait for the exchange.
//   combiner (warp 17)  waits on the exchange mbarrier for the kTmWarps * P
//            warp partials of a row, merges them with a fixed 32-lane
//            shuffle tree (the same arithmetic in every CTA, so the
//            statistics are bit-identical across the cluster) and publishes
//            them, up to two rows ahead of the writers.
//   writers  (warps 8-15)  wait for the row statistics, read the slice back
//            from TMEM (tcgen05.ld; writer thread w reads lane w % 128, half
//            w / 128, exactly what reducer thread w wrote), apply h and store
//            the output.  gamma / beta come from the shared-memory affine
//            ring or, when the rows' alignment does not allow staging, from L2.
//   A warp reaches only its TMEM lane quarter (warp % 4), which the mapping
//   above respects for every role.
//
// Capacity.  TMEM holds two row slices (two 256-column buffers, row parity),
// so a slice is at most kTmMaxChunks chunks: with 16 KiB chunks 128 KiB, the
// Eq. 3 capacity of this path.  A chunk stays in shared memory only from its
// landing to its sweep, so the ring needs no room for a whole slice and the
// rest of shared memory stages gamma / beta.  Row r is written from TMEM
// while row r + 1 is swept into the other buffer and row r + 2 streams into
// the ring; the exchange latency of a row overlaps the next row's sweep.
//
// Exchange slots and mbarriers are indexed by row % 4: a CTA's reducers reach
// row r + 4 only after its writers finished row r + 2, which needed every
// peer's row-(r + 2) partial, which each peer pushed only after its own
// writers had finished row r -- and those waited for the statistics its
// combiner computed from its row-r slots.  The push is ordered after those
// reads by a release fence restricted to shared memory at cluster scope; the
// combiner acquires at cluster scope.  TMEM buffers are indexed by row % 2 and
// handed back by the writers (tm_empty).
//
// One CTA per SM: the kernel allocates all 512 TMEM columns, and the host
// requests more than half of the SM's shared memory so no second CTA of this
// kernel can be resident on the SM (tcgen05.alloc then never waits).
#pragma once

#include "credit_rows.cuh"

namespace credit {

constexpr int kTmLanes = 128;                                  // TMEM lanes: lane t owns groups t + 128 i
constexpr int kTmGroups = 8;                                   // groups per lane per chunk
constexpr int kTmHalf = kTmGroups / 2;                         // groups per thread per chunk (two threads per lane)
constexpr int kTmReducers = 2 * kTmLanes;                      // warps 0-7
constexpr int kTmWriters = 2 * kTmLanes;                       // warps 8-15
constexpr int kTmThreads = kTmReducers + kTmWriters + 64;      // + producer (16) and combiner (17) warps
constexpr int kTmMaxChunkBytes = kTmLanes * kTmGroups * 16;    // 16 KiB
constexpr int kTmColsPerChunk = 4 * kTmGroups;                 // 32-bit columns per chunk and lane
constexpr int kTmCols = 512;                                   // allocated: two row buffers
constexpr int kTmBufCols = kTmCols / 2;
constexpr int kTmMaxChunks = kTmBufCols / kTmColsPerChunk;     // 8 chunks per slice
static_assert(kTmHalf * 4 == 16, "each thread stores / loads 16 columns per chunk");

constexpr int kTmCtrl = 9472;
constexpr int kTmWarps = kTmReducers / 32;  // reducer warps = partials per CTA and row

// Control area (kTmCtrl bytes):
//   [0, 256)       full[32] mbarriers (count 1 + transaction bytes)
//   [256, 512)     empty[32] mbarriers (count: reducer warps)
//   [512, 544)     exchange mbarriers [row % 4] (count 1 + kTmWarps, tx bytes)
//   [544, 560)     tm_empty[row % 2] mbarriers (count: writer warps)
//   [560, 564)     TMEM base address written by tcgen05.alloc
//   [576, 608)     stats_full[row % 4] mbarriers (count 1: the combiner)
//   [608, 640)     published row statistics [row % 4][2 floats]
//   [1024, 9216)   exchange slots [row % 4][16 CTAs][kTmWarps][4 floats]
//   [9216, 9280)   affine_full[8] mbarriers
//   [9280, 9344)   affine_empty[8] mbarriers
__device__ __forceinline__ float *tm_entry(float *slots, int s4, int c, int w) {
    return slots + ((s4 * 16 + c) * kTmWarps + w) * 4;
}

// Partial of one warp (or of the merge of several) as 4 floats:
//   softmax (m, s, -, -)   layernorm (mean, M2, n, -)   rmsnorm (sum x^2, -, -, -)
template <int OP> struct TmPart;
template <> struct TmPart<OP_SOFTMAX> {
    Stream<OP_SOFTMAX> st;
    __device__ __forceinline__ void from(const float4 &e) { st.m = e.x; st.s = e.y; }
    __device__ __forceinline__ float4 to() const { return make_float4(st.m, st.s, 0.0f, 0.0f); }
    __device__ __forceinline__ void merge(const TmPart &o) { st.merge(o.st.m, o.st.s); }
};
template <> struct TmPart<OP_LN> {
    Stream<OP_LN> st;
    __device__ __forceinline__ void from(const float4 &e) { st.mu = e.x; st.m2 = e.y; st.n = e.z; }
    __device__ __forceinline__ float4 to() const { return make_float4(st.mu, st.m2, st.n, 0.0f); }
    __device__ __forceinline__ void merge(const TmPart &o) { st.merge3(o.st.n, o.st.mu, o.st.m2); }
};
template <> struct TmPart<OP_RMS> {
    Stream<OP_RMS> st;
    __device__ __forceinline__ void from(const float4 &e) { st.ss = e.x; }
    __device__ __forceinline__ float4 to() const { return make_float4(st.ss, 0.0f, 0.0f, 0.0f); }
    __device__ __forceinline__ void merge(const TmPart &o) { st.ss += o.st.ss; }
};
template <> struct TmPart<OP_Q8> {
    Stream<OP_Q8> st;
    __device__ __forceinline__ void from(const float4 &e) { st.am = e.x; }
    __device__ __forceinline__ float4 to() const { return make_float4(st.am, 0.0f, 0.0f, 0.0f); }
    __device__ __forceinline__ void merge(const TmPart &o) { st.am = fmaxf(st.am, o.st.am); }
};

// Xor shuffle tree over the warp; both partners of a level merge (lower
// lane, upper lane) in that order, so every lane ends with the same value.
template <int OP>
__device__ __forceinline__ TmPart<OP> tm_warp_tree(TmPart<OP> t) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float4 e = t.to();
        float4 f = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        f.x = __shfl_xor_sync(0xffffffffu, e.x, o);
        if constexpr (OP != OP_RMS && OP != OP_Q8) f.y = __shfl_xor_sync(0xffffffffu, e.y, o);
        if constexpr (OP == OP_LN) f.z = __shfl_xor_sync(0xffffffffu, e.z, o);
        TmPart<OP> u;
        u.from(f);
        if (lane & o) {
            u.merge(t);
            t = u;
        } else {
            t.merge(u);
        }
    }
    return t;
}

template <int OP, int TIN, int TOUT>
__global__ void __launch_bounds__(kTmThreads, 1) k_ring_tm(const RowArgs a) {
    static_assert(OP != OP_LSE, "logsumexp writes no reuse pass");
    static_assert(!(TOUT == DT_E4M3 && (OP == OP_LN || OP == OP_RMS)), "FP8 norm output needs the amax stage");
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + 32;
    uint64_t *xbar = full + 64;
    uint64_t *tm_empty = full + 68;
    uint32_t *tm_base = reinterpret_cast<uint32_t *>(smem + 560);
    uint64_t *stats_full = reinterpret_cast<uint64_t *>(smem + 576);
    float *pub = reinterpret_cast<float *>(smem + 608);
    float *slots = reinterpret_cast<float *>(smem + 1024);
    uint64_t *affine_full = reinterpret_cast<uint64_t *>(smem + 9216);
    uint64_t *affine_empty = reinterpret_cast<uint64_t *>(smem + 9280);
    unsigned char *ring = smem + kTmCtrl;

    constexpr int isz = Fmt<TIN>::size, V = Fmt<TIN>::V;
    constexpr int SV = V < 8 ? V : 8;
    constexpr int osz = Fmt<TOUT>::size;
    constexpr int Tr = kTmReducers, Tw = kTmWriters, TL = kTmLanes;

    const int CH = a.chunk_bytes, K = a.ring, gpc = CH / 16;
    const int A = a.affine;
    const bool has_g = a.gamma != nullptr, has_b = (OP == OP_LN) && a.beta != nullptr;
    const int aseg = gpc * V * 4;
    const int aslot = aseg * ((has_g ? 1 : 0) + (has_b ? 1 : 0));
    unsigned char *aring = ring + static_cast<size_t>(K) * CH;
    const int P = static_cast<int>(cluster_nctarank());
    const int c = P > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const long long ncl = gridDim.x / P, cl = blockIdx.x / P;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long N = a.cols;

    if (tid == 0) {
        for (int k = 0; k < K; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], static_cast<uint32_t>(Tr / 32));
        }
        for (int k = 0; k < 4; ++k) {
            mbar_init(&xbar[k], 1 + kTmWarps);
            mbar_init(&stats_full[k], 1);
        }
        for (int k = 0; k < 2; ++k) mbar_init(&tm_empty[k], static_cast<uint32_t>(Tw / 32));
        for (int k = 0; k < A; ++k) {
            mbar_init(&affine_full[k], 1);
            mbar_init(&affine_empty[k], static_cast<uint32_t>(Tw / 32));
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        tm_alloc(tm_base, kTmCols);
        tm_relinquish();
    }
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    const uint32_t taddr = *tm_base;
    // this warp's lane quarter (reducer warps q, 4 + q and writer warps 8 + q, 12 + q share it)
    const uint32_t tq = taddr + ((static_cast<uint32_t>(warp & 3) * 32u) << 16);
    if (P > 1) cluster_arrive_release();  // start barrier, split
    bool waited_start = false;

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
    auto chunk_groups = [&](const RowGeo &g, int k) -> int {
        const long long r = g.ng - static_cast<long long>(k) * gpc;
        return static_cast<int>(r < gpc ? r : gpc);
    };
    auto edge_x = [&](const RowGeo &g, int e, long long k) -> float {
        const long long i = e == 0 ? k : g.s.h0 + g.s.G * V + k;
        return decode_one<TIN>(g.in_row + i * isz, g.in_sc);
    };

    if (warp == 17) {
        // ========================================================== combiner
        // Row r's statistics land in pub[r % 4] once xbar[r % 4] completes;
        // that completion needs this CTA's own push of row r, made after its
        // writers finished row r - 2, so the writers no longer read pub[r % 4]
        // (they last read it for row r - 4).
        const int ne = P * kTmWarps;  // warp partials per row, entry e = c * kTmWarps + w
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const int s4 = rr & 3;
            if (lane == 0)
                mbar_arrive_expect_tx(&xbar[s4], static_cast<uint32_t>((P - 1) * kTmWarps * 16));
            mbar_wait_bounded_cluster(&xbar[s4], static_cast<uint32_t>((rr >> 2) & 1), a.err);
            TmPart<OP> t;
            if (lane < ne) t.from(*reinterpret_cast<const float4 *>(slots + (s4 * 16 * kTmWarps + lane) * 4));
#pragma unroll
            for (int e = lane + 32; e < 16 * kTmWarps; e += 32) {
                if (e < ne) {
                    TmPart<OP> u;
                    u.from(*reinterpret_cast<const float4 *>(slots + (s4 * 16 * kTmWarps + e) * 4));
                    t.merge(u);
                }
            }
            t = tm_warp_tree<OP>(t);
            if (lane == 0) {
                Stats st;
                if constexpr (OP == OP_SOFTMAX) {
                    st.a = t.st.m;
                    st.b = t.st.s;
                } else if constexpr (OP == OP_LN) {
                    st.a = t.st.mu;
                    st.b = rsqrtf(t.st.m2 / static_cast<float>(N) + a.eps);
                } else if constexpr (OP == OP_Q8) {
                    st.a = t.st.am > 0.0f ? __fdiv_rn(t.st.am, 127.0f) : 1.0f;  // the row scale
                    st.b = __frcp_rn(st.a);
                    if (c == 0) a.out_scale[row] = st.a;
                } else {
                    st.a = rsqrtf(t.st.ss / static_cast<float>(N) + a.eps);
                    st.b = 0.0f;
                }
                pub[s4 * 2] = st.a;
                pub[s4 * 2 + 1] = st.b;
                mbar_arrive(&stats_full[s4]);
            }
            __syncwarp();
        }
    } else if (warp == 16) {
        // ========================================================== producer
        if (lane == 0) {
            RingPos rp(K);
            for (long long row = cl; row < a.rows; row += ncl) {
                const RowGeo g = geo(row);
                const long long body = g.ng * 16;
                const unsigned char *src = g.in_row + g.s.h0 * isz + g.s.g_lo * 16;
                for (long long off = 0; off < body; off += CH, rp.next()) {
                    const int slot = rp.slot;
                    if (rp.lap > 0) mbar_wait_bounded(&empty[slot], rp.prev_parity(), a.err);
                    const uint32_t bytes = static_cast<uint32_t>(body - off < CH ? body - off : CH);
                    mbar_arrive_expect_tx(&full[slot], bytes);
                    bulk_g2s(ring + static_cast<size_t>(slot) * CH, src + off, bytes, &full[slot]);
                }
            }
        } else if (lane == 1 && A > 0) {
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
    } else if (warp < Tr / 32) {
        // ========================================================== reducers
        // reducer thread tid owns lane t = tid % 128 and the half tid / 128 of
        // that lane's groups in every chunk: groups t + 128 (4 half + m)
        const int t = tid & (TL - 1), half = tid / TL;
        RingPos rp(K);
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const RowGeo g = geo(row);
            const int b = rr & 1, s4 = rr & 3;
            if (tid == 0) trace_stamp(a, rr, 0);
            if (rr >= 2) {
                mbar_wait_bounded(&tm_empty[b], static_cast<uint32_t>(((rr >> 1) - 1) & 1), a.err);
                tm_fence_after();
            }
            if (tid == 0) trace_stamp(a, rr, 5);
            const uint32_t tb = tq + static_cast<uint32_t>(b * kTmBufCols + half * 4 * kTmHalf);
            Stream<OP> acc;
            for (int k = 0; k < g.nch; ++k, rp.next()) {
                const int slot = rp.slot;
                mbar_wait_bounded(&full[slot], rp.parity(), a.err);
                const unsigned char *cb = ring + static_cast<size_t>(slot) * CH;
                const int gn = chunk_groups(g, k);
                const int g0 = t + half * kTmHalf * TL;
                uint32_t w[4 * kTmHalf];
#pragma unroll
                for (int m = 0; m < kTmHalf; ++m) {
                    const int gi = g0 + m * TL;
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (gi < gn) v = *reinterpret_cast<const uint4 *>(cb + gi * 16);
                    w[4 * m] = v.x;
                    w[4 * m + 1] = v.y;
                    w[4 * m + 2] = v.z;
                    w[4 * m + 3] = v.w;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
#pragma unroll
                for (int m = 0; m < kTmHalf; ++m)
                    if (g0 + m * TL < gn)
                        stream_add_group<OP, TIN>(acc, make_uint4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]),
                                                  g.in_sc);
                tm_st16_issue(tb + static_cast<uint32_t>(k * kTmColsPerChunk), w);
            }
            tm_wait_st();  // the row's TMEM stores, complete before the handoff below
            // edge elements, one per reducer thread (head element tid, tail element Tr - 1 - tid)
            if (c == 0 && tid < g.s.h0) acc.add1(edge_x(g, 0, tid));
            if (c == P - 1 && Tr - 1 - tid < g.s.t0) acc.add1(edge_x(g, 1, Tr - 1 - tid));
            if (tid == 0) trace_stamp(a, rr, 1);
            // ---------- warp partial, pushed to every CTA of the cluster (Eq. 5)
            if constexpr (OP == OP_LN) acc.finish();
            TmPart<OP> part;
            part.st = acc;
            part = tm_warp_tree<OP>(part);
            const float4 e = part.to();
            if (tid == 0) trace_stamp(a, rr, 2);
            if (P > 1 && !waited_start) {
                cluster_wait_acquire();
                waited_start = true;
            }
            float *ent = tm_entry(slots, s4, c, warp);
            tm_fence_before();  // this warp's TMEM stores, before its arrival below
            __syncwarp();
            if (lane == 0) {
                *reinterpret_cast<float4 *>(ent) = e;
                mbar_arrive(&xbar[s4]);
            } else if (lane < P) {
                const uint32_t d = static_cast<uint32_t>((c + lane) % P);
                fence_release_smem_cluster();
                st_async_v4f32(mapa_shared(smem_addr(ent), d), e, mapa_shared(smem_addr(&xbar[s4]), d));
            }
        }
    } else {
        // ========================================================== writers
        const int wt = tid - Tr;
        const int twin = wt & (TL - 1), half = wt / TL;  // the lane, and the half of its groups (as the reducers)
        RingPos wa(A > 0 ? A : 1);  // streamed gamma / beta slots
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const RowGeo g = geo(row);
            const int b = rr & 1, s4 = rr & 3;
            if (wt == 0) trace_stamp(a, rr, 6);
            mbar_wait_bounded(&stats_full[s4], static_cast<uint32_t>((rr >> 2) & 1), a.err);
            Stats st;
            st.a = pub[s4 * 2];
            st.b = pub[s4 * 2 + 1];
            tm_fence_after();
            if (wt == 0) trace_stamp(a, rr, 3);
            if constexpr (OP == OP_SOFTMAX && TOUT == DT_E4M3) {
                if (c == 0 && wt == 0) a.out_scale[row] = (1.0f / st.b) * (1.0f / 448.0f);
            }
            unsigned char *out_row = a.out + row * a.ld_out * osz;
            const long long i_base = g.s.h0 + g.s.g_lo * V;
            constexpr int vec_bytes = (SV * osz) < 16 ? (SV * osz) : 16;
            const bool out_vec = ((reinterpret_cast<uintptr_t>(out_row) + g.s.h0 * osz) % vec_bytes) == 0;
            const bool g_vec = a.gamma == nullptr || ((reinterpret_cast<uintptr_t>(a.gamma + g.s.h0) & 15u) == 0);
            const bool b_vec = a.beta == nullptr || ((reinterpret_cast<uintptr_t>(a.beta + g.s.h0) & 15u) == 0);
            const float smul = (TOUT == DT_E4M3) ? 448.0f : ((OP == OP_SOFTMAX) ? 1.0f / st.b : 0.0f);
            // softmax: y (or its FP8 code) = exp(x - M) * smul = 2^((x - M) log2 e + log2 smul)
            const float cL = (OP == OP_SOFTMAX) ? log2f(smul) : 0.0f;  // exp_sub's log2-domain scale
            auto h = [&](float x, float gm, float bt) -> float {
                if constexpr (OP == OP_SOFTMAX) return exp_sub(x, st.a, cL);
                else if constexpr (OP == OP_Q8) return q8_code(x, st.a, st.b);
                else return norm_h<OP>(x, st, gm, bt);
            };
            const uint32_t tb = tq + static_cast<uint32_t>(b * kTmBufCols);
            for (int k = 0; k < g.nch; ++k) {
                const int gn = chunk_groups(g, k);
                const long long kg = static_cast<long long>(k) * gpc;
                const int aslot_k = A > 0 ? (a.affine_resident ? k : wa.slot) : 0;
                const float *ag = reinterpret_cast<const float *>(aring + static_cast<size_t>(aslot_k) * aslot);
                const float *ab = ag + (has_g ? gpc * V : 0);
                if (A > 0 && (!a.affine_resident || rr == 0))
                    mbar_wait_bounded(&affine_full[aslot_k], a.affine_resident ? 0u : wa.parity(), a.err);
                uint32_t w[4 * kTmHalf];
                tm_ld16(tb + static_cast<uint32_t>(k * kTmColsPerChunk + half * 4 * kTmHalf), w);
                // Fast path: every one of this thread's kTmHalf groups lies in the chunk (its last one,
                // twin + (half * kTmHalf + kTmHalf - 1) * TL, is below gn; a chunk can hold fewer than
                // TL * kTmGroups groups), vector stores, gamma / beta (where the op has them) staged in shared
                // memory -- no per-group bounds or pointer tests, 32-bit offsets from the chunk's output base.
                constexpr bool kNormOp = OP == OP_LN || OP == OP_RMS;
                const bool fast = out_vec && twin + (half * kTmHalf + kTmHalf - 1) * TL < gn &&
                                  (!kNormOp || (A > 0 && has_g && (OP != OP_LN || has_b)));
                if (fast) {
                    unsigned char *oc = out_row + (i_base + kg * V) * osz;
                    float gg[kTmHalf][kNormOp ? V : 1], bb[kTmHalf][OP == OP_LN ? V : 1];
                    if constexpr (kNormOp) {
#pragma unroll
                        for (int m = 0; m < kTmHalf; ++m) {
                            const int gi = twin + (half * kTmHalf + m) * TL;
                            lds_f32<V>(ag + gi * V, gg[m]);
                            if constexpr (OP == OP_LN) lds_f32<V>(ab + gi * V, bb[m]);
                        }
                    }
                    // E4M3 softmax codes from the raw input codes (softmax_e4m3_codes) with 16-byte stores,
                    // where the output groups start on the 16-byte grid (out_vec checks 8 bytes here)
                    constexpr bool kRaw8 = OP == OP_SOFTMAX && TIN == DT_E4M3 && TOUT == DT_E4M3;
                    const bool raw8 = kRaw8 && ((reinterpret_cast<uintptr_t>(out_row) + g.s.h0) & 15u) == 0;
                    if (raw8) {
                        const uint32_t neg = e4m3_sign_mask(g.in_sc);
                        const float a1 = fabsf(g.in_sc);
#pragma unroll
                        for (int m = 0; m < kTmHalf; ++m) {
                            const int gi = twin + (half * kTmHalf + m) * TL;
                            *reinterpret_cast<uint4 *>(oc + static_cast<uint32_t>(gi * V)) = softmax_e4m3_codes(
                                e4m3_fold_sign(make_uint4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]), neg),
                                a1, st.a);
                        }
                    } else {
#pragma unroll
                    for (int m = 0; m < kTmHalf; ++m) {
                        const int gi = twin + (half * kTmHalf + m) * TL;
                        float f[V];
                        decode_group<TIN>(make_uint4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]), f, g.in_sc);
#pragma unroll
                        for (int hv = 0; hv < V; hv += SV) {
                            float y[SV];
                            if constexpr (OP == OP_Q8) {
                                float xs[SV];
#pragma unroll
                                for (int q = 0; q < SV; ++q) xs[q] = f[hv + q];
                                q8_codes<SV>(xs, st.a, st.b, y);
                            } else if constexpr (OP == OP_SOFTMAX) {  // h on element pairs (the same bits as h)
                                float xs[SV];
#pragma unroll
                                for (int q = 0; q < SV; ++q) xs[q] = f[hv + q];
                                exp_sub_group<SV>(xs, st.a, cL, y);
                            } else {
#pragma unroll
                                for (int q = 0; q < SV; ++q)
                                    y[q] = h(f[hv + q], kNormOp ? gg[m][kNormOp ? hv + q : 0] : 1.0f,
                                             OP == OP_LN ? bb[m][OP == OP_LN ? hv + q : 0] : 0.0f);
                            }
                            store_group<TOUT, SV>(oc + static_cast<uint32_t>((gi * V + hv) * osz), y, true);
                        }
                    }
                    }
                } else {
                // gamma / beta for the groups of this chunk, batch by batch (L2 loads issued together)
                constexpr int MB = (V == 4) ? 4 : (V == 8 ? 2 : 1);
#pragma unroll
                for (int m0 = 0; m0 < kTmHalf; m0 += MB) {
                    float gg[MB][V], bb[MB][V];
#pragma unroll
                    for (int u = 0; u < MB; ++u) {
                        const int gi = twin + (half * kTmHalf + m0 + u) * TL;
                        const long long i0 = i_base + (kg + gi) * V;
#pragma unroll
                        for (int hv = 0; hv < V; hv += SV) {
                            float tg[SV], tbv[SV];
                            if constexpr (OP == OP_LN || OP == OP_RMS) {
                                if (gi < gn) {
                                    if (A > 0) {
                                        load_affine_smem<SV>(has_g ? ag : nullptr, gi * V + hv, 1.0f, tg);
                                        load_affine_smem<SV>(has_b ? ab : nullptr, gi * V + hv, 0.0f, tbv);
                                    } else {
                                        load_affine<SV>(has_g ? a.gamma : nullptr, i0 + hv, g_vec, 1.0f, tg);
                                        load_affine<SV>(has_b ? a.beta : nullptr, i0 + hv, b_vec, 0.0f, tbv);
                                    }
                                } else {
#pragma unroll
                                    for (int q = 0; q < SV; ++q) {
                                        tg[q] = 1.0f;
                                        tbv[q] = 0.0f;
                                    }
                                }
                            } else {
#pragma unroll
                                for (int q = 0; q < SV; ++q) {
                                    tg[q] = 1.0f;
                                    tbv[q] = 0.0f;
                                }
                            }
#pragma unroll
                            for (int q = 0; q < SV; ++q) {
                                gg[u][hv + q] = tg[q];
                                bb[u][hv + q] = tbv[q];
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < MB; ++u) {
                        const int m = m0 + u;
                        const int gi = twin + (half * kTmHalf + m) * TL;
                        if (gi >= gn) continue;
                        float f[V];
                        decode_group<TIN>(make_uint4(w[4 * m], w[4 * m + 1], w[4 * m + 2], w[4 * m + 3]), f, g.in_sc);
                        const long long i0 = i_base + (kg + gi) * V;
#pragma unroll
                        for (int hv = 0; hv < V; hv += SV) {
                            float y[SV];
#pragma unroll
                            for (int q = 0; q < SV; ++q) y[q] = h(f[hv + q], gg[u][hv + q], bb[u][hv + q]);
                            store_group<TOUT, SV>(out_row + (i0 + hv) * osz, y, out_vec);
                        }
                    }
                }
                }
                if (A > 0 && !a.affine_resident) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&affine_empty[aslot_k]);
                    wa.next();
                }
            }
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
            tm_fence_before();  // this warp's TMEM loads, before handing the buffer back
            __syncwarp();
            if (lane == 0) mbar_arrive(&tm_empty[b]);
            if (wt == 0) trace_stamp(a, rr, 4);
        }
    }
    // release TMEM once every warp is done with it, then the end barrier
    tm_fence_before();
    __syncthreads();
    if (warp == 0) {
        tm_fence_after();
        tm_dealloc(taddr, kTmCols);
    }
    if (P > 1) {
        if (!waited_start) cluster_wait_acquire();
        cluster_arrive_release();  // nobody exits while a peer may push into it
        cluster_wait_acquire();
    }
}

}  // namespace credit
