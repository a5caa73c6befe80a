// credit_ragged.cu -- ragged batches: rows of uneven width and mixed op
// (softmax / RMSNorm) in one persistent cluster launch, captured in a CUDA
// graph, with the launch shape chosen by timing the batch (autotuner).
//
// Work items, built on the host from the row list (widest first, dealt
// round-robin to the persistent clusters):
//   staged  P / w rows, each split over w CTAs of the cluster (w = 1, 2, 4,
//           ..., P: the smallest power of two whose slices fit one CTA's
//           staging capacity; Eq. 2-3): every slice staged once in shared
//           memory, the partials of a row exchanged over DSMEM among its w
//           CTAs (Eq. 5), the output written from shared memory.  w = 1 is
//           the one-CTA path, w = P the cluster path of one row.
//   huge    a row whose slices exceed the staging capacity even over all P
//           CTAs: each CTA streams its part through the staging buffer as a
//           ring of bulk-copied chunks, the partials are exchanged, then the
//           part is written: first the chunks the ring still holds, then the
//           rest, read again (the two-pass schedule inside a cluster)
// While a CTA writes a staged item, every chunk slot it has written out takes
// the same chunk of the CTA's slice of its next item (a bulk copy issued at
// once), so the loads of item i + 1 overlap the writes of item i; a next item
// that streams is moved towards L2 instead.
// Exchanges among changing subsets of the cluster: a CTA's slots are reused
// by every item that exchanges (w > 1 or huge), so each such item ends with a
// split cluster barrier that every CTA executes (arrive once it has read its
// slots, wait before the next exchanging item's pushes; items of width 1
// exchange nothing and skip it); each CTA tracks the phase of its own
// exchange mbarrier.
// The op is a per-row field; the element type is a template parameter.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_rows.cuh"

namespace credit {
extern std::atomic<long long> g_launch_count;
}

using namespace credit;

namespace {

enum : int { ITEM_STAGED = 0, ITEM_HUGE = 2 };

struct RRow {
    long long in_off, out_off, cols;  // elements
    int op;
    int pad;
};
struct RItem {
    int kind;
    int count;      // staged: rows in the item (<= P / width)
    long long row;  // first row (index into the row table)
    int width;      // staged: CTAs per row (a power of two <= P); huge: P
    int pad;
};
struct RaggedArgs {
    const unsigned char *in;
    unsigned char *out;
    const RRow *rows;
    const RItem *items;
    long long n_items;
    int cap;  // staging capacity per CTA (bytes, multiple of the chunk size)
    float eps;
    unsigned *err;
};

constexpr int kRCtrl = 1280;  // [0,128) mbarriers, [128,384) slots [16][4], [640,1152) reduction scratch (128 floats)
constexpr int kRChunk = 16384;

// Groups gb .. ge - 1 of a staged buffer, VW per thread per step (the
// vector width the autotuner picks: VW independent 16-byte reads in flight
// before any is used): fn(group, its 16 bytes).
template <int VW, class F>
__device__ __forceinline__ void for_groups(const unsigned char *base, long long gb, long long ge, int tid, int T,
                                           F &&fn) {
    for (long long g = gb + tid; g < ge; g += static_cast<long long>(VW) * T) {
        uint4 w[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u)
            if (g + static_cast<long long>(u) * T < ge) w[u] = *reinterpret_cast<const uint4 *>(base + (g + u * T) * 16);
#pragma unroll
        for (int u = 0; u < VW; ++u)
            if (g + static_cast<long long>(u) * T < ge) fn(g + static_cast<long long>(u) * T, w[u]);
    }
}

template <int TIN, int VW>
__device__ __forceinline__ float2 stats_from_smem(int op, const unsigned char *buf, long long ng, const RowSlice &s,
                                                  bool own_head, bool own_tail, const unsigned char *row,
                                                  uint64_t *mbar, uint32_t &phase_bits, int nch, float *red,
                                                  unsigned *err) {
    constexpr int V = Fmt<TIN>::V, isz = Fmt<TIN>::size;
    const int tid = threadIdx.x, T = blockDim.x;
    Stream<OP_SOFTMAX> sm;
    Stream<OP_RMS> rs;
    for (int k = 0; k < nch; ++k) {
        mbar_wait_bounded(&mbar[k], (phase_bits >> k) & 1u, err);
        const long long gb = static_cast<long long>(k) * (kRChunk / 16);
        const long long ge = min(ng, gb + kRChunk / 16);
        for_groups<VW>(buf, gb, ge, tid, T, [&](long long, const uint4 &w) {
            float f[V];
            decode_group<TIN>(w, f, 1.0f);
            if (op == OP_SOFTMAX) sm.add(f);
            else rs.add(f);
        });
    }
    phase_bits ^= (nch >= 32 ? 0xFFFFFFFFu : ((1u << nch) - 1u));
    // edge elements, one per thread: head element tid, tail element T - 1 - tid
    for (int e = 0; e < 2; ++e) {
        const long long i = e == 0 ? ((own_head && tid < s.h0) ? tid : -1)
                                   : ((own_tail && T - 1 - tid < s.t0) ? s.h0 + s.G * V + (T - 1 - tid) : -1);
        if (i < 0) continue;
        const float x = decode_one<TIN>(row + i * isz, 1.0f);
        if (op == OP_SOFTMAX) sm.add1(x);
        else rs.add1(x);
    }
    if (op == OP_SOFTMAX) return block_reduce_stream<OP_SOFTMAX>(sm, red, 0);
    return block_reduce_stream<OP_RMS>(rs, red, 0);
}

// Exchange among the w CTAs of a row (ranks base .. base + w - 1 of the
// cluster; this CTA is number cs of them): every thread returns the combined
// statistics.  Partial of CTA cs lands in slot cs of each of them, pushed
// with st.async onto the receiver's exchange mbarrier (Eq. 5); xph is this
// CTA's phase of that mbarrier.  The caller's per-item cluster barrier keeps
// the next item's pushes behind this combine's reads of the slots.
template <int TIN>
__device__ __forceinline__ Stats exchange_sub(int op, float2 part, float *slots, uint64_t *xbar, uint32_t &xph,
                                             int base, int w, int cs, const RowSlice &s, long long N, float eps,
                                             unsigned *err) {
    constexpr int V = Fmt<TIN>::V;
    Stats st;
    if (w > 1) {
        const int tid = threadIdx.x;
        float *mine = slots + cs * 4;
        if (tid < w) {
            if (tid == cs) {
                mine[0] = part.x;
                mine[1] = part.y;
            } else {
                fence_release_smem_cluster();  // this CTA's earlier reads of the slots first
                const uint32_t peer = static_cast<uint32_t>(base + tid);
                st_async_v2f32(mapa_shared(smem_addr(mine), peer), part.x, part.y, mapa_shared(smem_addr(xbar), peer));
            }
        }
        if (tid == 0) mbar_arrive_expect_tx(xbar, static_cast<uint32_t>((w - 1) * 8));
        __syncthreads();
        mbar_wait_bounded_cluster(xbar, xph, err);
        xph ^= 1u;
        st = op == OP_SOFTMAX ? combine_partials<OP_SOFTMAX>(slots, 4, w, s, V, N, eps)
                              : combine_partials<OP_RMS>(slots, 4, w, s, V, N, eps);
    } else {
        const float p1[2] = {part.x, part.y};
        st = op == OP_SOFTMAX ? combine_partials<OP_SOFTMAX>(p1, 2, 1, s, V, N, eps)
                              : combine_partials<OP_RMS>(p1, 2, 1, s, V, N, eps);
    }
    return st;
}

// Stream ng 16-byte groups from src (16-byte aligned) through buf as a ring of
// R chunk slots: thread 0 keeps up to R bulk copies in flight and refills a
// slot once every thread is done with it; fn(first group, groups, slot) runs
// on every chunk in order.  The chunk barriers and their phases (phase_bits)
// are the ones the staged items use.
template <class F>
__device__ __forceinline__ void ring_stream(const unsigned char *src, long long ng, unsigned char *buf, int R,
                                            uint64_t *mbar, uint32_t &phase_bits, unsigned *err, uint64_t policy,
                                            F &&fn) {
    const long long body = ng * 16;
    const long long nch = (body + kRChunk - 1) / kRChunk;
    auto issue = [&](long long k, int slot) {
        const long long off = k * kRChunk;
        const uint32_t bytes = static_cast<uint32_t>(min(static_cast<long long>(kRChunk), body - off));
        mbar_arrive_expect_tx(&mbar[slot], bytes);
        bulk_g2s_hint(buf + static_cast<size_t>(slot) * kRChunk, src + off, bytes, &mbar[slot], policy);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < R && k < nch; ++k) issue(k, k);
    int slot = 0;
    for (long long k = 0; k < nch; ++k) {
        mbar_wait_bounded(&mbar[slot], (phase_bits >> slot) & 1u, err);
        phase_bits ^= 1u << slot;
        const long long g0 = k * (kRChunk / 16);
        fn(g0, static_cast<int>(min(static_cast<long long>(kRChunk / 16), ng - g0)),
           buf + static_cast<size_t>(slot) * kRChunk);
        __syncthreads();  // the slot's data has been used by every thread
        if (threadIdx.x == 0 && k + R < nch) issue(k + R, slot);
        if (++slot == R) slot = 0;
    }
}

// The second pass over a part that ring_stream has just streamed: its last
// min(R, nch) chunks are still in their slots (chunk k in slot k % R), so
// they are used first, without a copy, and each slot they free takes one of
// the chunks that are read again.  Those go newest first (chunk again - 1
// down to 0, the i-th into slot (nch + i) % R): the most recently read lines
// are the likeliest to be still in L2.
template <class F>
__device__ __forceinline__ void ring_stream_again(const unsigned char *src, long long ng, unsigned char *buf, int R,
                                                  uint64_t *mbar, uint32_t &phase_bits, unsigned *err,
                                                  uint64_t policy, F &&fn) {
    const long long body = ng * 16;
    const long long nch = (body + kRChunk - 1) / kRChunk;
    const long long kept = min(static_cast<long long>(R), nch), again = nch - kept;
    auto slot_of = [&](long long k) { return static_cast<int>(k % R); };
    auto issue = [&](long long i) {  // the i-th chunk read again: chunk again - 1 - i
        const int slot = static_cast<int>((nch + i) % R);
        const long long off = (again - 1 - i) * kRChunk;
        const uint32_t bytes = static_cast<uint32_t>(min(static_cast<long long>(kRChunk), body - off));
        mbar_arrive_expect_tx(&mbar[slot], bytes);
        bulk_g2s_hint(buf + static_cast<size_t>(slot) * kRChunk, src + off, bytes, &mbar[slot], policy);
    };
    long long next = 0;  // the next chunk to read again
    for (long long k = nch - kept; k < nch; ++k) {
        const long long g0 = k * (kRChunk / 16);
        fn(g0, static_cast<int>(min(static_cast<long long>(kRChunk / 16), ng - g0)),
           buf + static_cast<size_t>(slot_of(k)) * kRChunk);
        __syncthreads();
        if (threadIdx.x == 0 && next < again) issue(next);
        ++next;
    }
    for (long long i = 0; i < again; ++i) {
        const int slot = static_cast<int>((nch + i) % R);
        mbar_wait_bounded(&mbar[slot], (phase_bits >> slot) & 1u, err);
        phase_bits ^= 1u << slot;
        const long long g0 = (again - 1 - i) * (kRChunk / 16);
        fn(g0, static_cast<int>(min(static_cast<long long>(kRChunk / 16), ng - g0)),
           buf + static_cast<size_t>(slot) * kRChunk);
        __syncthreads();
        if (threadIdx.x == 0 && i + R < again) issue(i + R);
    }
}

template <int TIN>
__device__ __forceinline__ float h_of(int op, float x, const Stats &st, float inv) {
    return op == OP_SOFTMAX ? exp_fast(x - st.a) * inv : x * st.a;
}
// h_of over one decoded group, two elements per packed f32x2 subtraction and multiply (the same bits as
// h_of element by element), the op tested once per group.
template <int V>
__device__ __forceinline__ void h_group(int op, const float (&f)[V], const Stats &st, float inv, float (&y)[V]) {
    static_assert(V % 2 == 0, "groups hold an even number of elements");
    if (op == OP_SOFTMAX) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float2 t = __fmul2_rn(__fadd2_rn(make_float2(f[j], f[j + 1]), make_float2(-st.a, -st.a)),
                                        make_float2(kLog2e, kLog2e));
            const float2 e = __fmul2_rn(make_float2(ex2_approx(t.x), ex2_approx(t.y)), make_float2(inv, inv));
            y[j] = e.x;
            y[j + 1] = e.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float2 e = __fmul2_rn(make_float2(f[j], f[j + 1]), make_float2(st.a, st.a));
            y[j] = e.x;
            y[j + 1] = e.y;
        }
    }
}

// This CTA's slice of a later item, moved from HBM into L2 while the current
// item is written (at most the staging capacity), so that its bulk copies
// find it there.
__device__ __forceinline__ void prefetch_next(const RaggedArgs &a, const RItem &nx, int P, int c, int isz) {
    const bool huge = nx.kind == ITEM_HUGE;
    const int w = huge ? P : nx.width;
    const int sub = c / w, cs = c % w;
    if (!huge && sub >= nx.count) return;
    const RRow rw = a.rows[nx.row + (huge ? 0 : sub)];
    const unsigned char *row = a.in + rw.in_off * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(row), rw.cols, isz, w, cs);
    const long long bytes = min((s.g_hi - s.g_lo) * 16, static_cast<long long>(a.cap));
    if (bytes > 0) bulk_prefetch_l2(row + s.h0 * isz + s.g_lo * 16, static_cast<uint32_t>(bytes));
}

// Where this CTA's slice of a staged item lies (16-byte aligned start, bytes, chunks); false when the CTA has
// no row in the item.
struct SliceSrc {
    const unsigned char *src;
    uint32_t body;
    int nch;
};
__device__ __forceinline__ bool staged_slice_of(const RaggedArgs &a, const RItem &it, int c, int isz, SliceSrc &o) {
    const int w = it.width, sub = c / w, cs = c % w;
    if (sub >= it.count) return false;
    const RRow rw = a.rows[it.row + sub];
    const unsigned char *row = a.in + rw.in_off * isz;
    const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(row), rw.cols, isz, w, cs);
    o.src = row + s.h0 * isz + s.g_lo * 16;
    o.body = static_cast<uint32_t>((s.g_hi - s.g_lo) * 16);
    o.nch = static_cast<int>((o.body + kRChunk - 1) / kRChunk);
    return true;
}
// A staged slice is read once: its lines go first when L2 needs room, so
// that a streamed part's lines stay for their second read.
__device__ __forceinline__ void issue_chunk(unsigned char *buf, const SliceSrc &sl, int k, uint64_t *mbar) {
    const uint32_t off = static_cast<uint32_t>(k) * kRChunk;
    const uint32_t bytes = min(static_cast<uint32_t>(kRChunk), sl.body - off);
    mbar_arrive_expect_tx(&mbar[k], bytes);
    bulk_g2s_hint(buf + off, sl.src + off, bytes, &mbar[k], l2_evict_first_policy());
}

// VW = 1 fits 64 registers (4 CTAs of 256 threads per SM); VW = 2 keeps two
// groups' registers live and is built for 2 CTAs per SM: the autotuner
// weighs the wider steps against the occupancy they cost.
template <int TIN, int VW>
__global__ void __launch_bounds__(256, VW == 2 ? 2 : 4) k_ragged(const RaggedArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem);       // [0..14) chunks, [14] exchange
    uint64_t *xbar = mbar + 14;
    float *slots = reinterpret_cast<float *>(smem + 128);
    float *red = reinterpret_cast<float *>(smem + 640);
    unsigned char *buf = smem + kRCtrl;
    constexpr int isz = Fmt<TIN>::size, V = Fmt<TIN>::V;
    const int P = static_cast<int>(cluster_nctarank());
    const int c = P > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const long long ncl = gridDim.x / P, cl = blockIdx.x / P;
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) {
        for (int k = 0; k < 16; ++k) mbar_init(&mbar[k], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (P > 1) {
        cluster_arrive_release();
        cluster_wait_acquire();  // peers' exchange barriers are initialised
    }
    uint32_t phase_bits = 0, xph = 0;
    bool pending = false;  // this CTA has arrived on the per-item cluster barrier and not yet waited
    int pre_issued = 0;    // thread 0: chunks of this item already requested while the previous one was written
    for (long long it = cl; it < a.n_items; it += ncl) {
        const RItem item = a.items[it];
        const bool huge = item.kind == ITEM_HUGE;
        const int w = huge ? P : item.width;      // CTAs per row
        const bool xch = P > 1 && (huge || w > 1);  // this item exchanges partials over DSMEM
        if (xch && pending) {  // every CTA has read its slots of the last exchanging item: pushes may follow
            cluster_wait_acquire();
            pending = false;
        }
        const int sub = c / w, cs = c % w;        // which row of the item, and which slice of it
        const bool active = huge || sub < item.count;
        const long long ri = item.row + (huge ? 0 : sub);
        const RRow rw = a.rows[active ? ri : item.row];
        const int op = rw.op;
        const long long N = rw.cols;
        const unsigned char *row = a.in + rw.in_off * isz;
        unsigned char *orow = a.out + rw.out_off * isz;
        const int Pslice = w;
        const int cslice = cs;
        const RowSlice s = make_slice(reinterpret_cast<uintptr_t>(row), N, isz, Pslice, cslice);
        const long long ng = s.g_hi - s.g_lo;
        const bool own_head = cslice == 0, own_tail = cslice == Pslice - 1;
        const long long i_base = s.h0 + s.g_lo * V;
        const bool out_vec = ((reinterpret_cast<uintptr_t>(orow) + s.h0 * isz) & 15u) == 0;
        if (item.kind != ITEM_HUGE) {
            // ---- staged: TMA the slice into shared memory (chunks), reduce, [exchange], write
            const SliceSrc cur{row + s.h0 * isz + s.g_lo * 16, static_cast<uint32_t>(ng * 16),
                               active ? static_cast<int>((ng * 16 + kRChunk - 1) / kRChunk) : 0};
            const int nch = cur.nch;
            __syncthreads();  // the previous item's reads of buf are done
            if (tid == 0)
                for (int k = pre_issued; k < nch; ++k) issue_chunk(buf, cur, k, mbar);
            pre_issued = 0;
            float2 part = make_float2(op == OP_SOFTMAX ? -INFINITY : 0.0f, 0.0f);
            if (active)
                part = stats_from_smem<TIN, VW>(op, buf, ng, s, own_head, own_tail, row, mbar, phase_bits, nch, red,
                                            a.err);
            Stats st{};
            if (active) st = exchange_sub<TIN>(op, part, slots, xbar, xph, sub * w, w, cs, s, N, a.eps, a.err);
            if (xch) {  // this CTA's slot reads are done
                cluster_arrive_release();
                pending = true;
            }
            // the next item: a staged slice is requested chunk by chunk as the slots free up below, a huge
            // part is moved towards L2
            SliceSrc nx{};
            bool pre = false;
            if (tid == 0 && it + ncl < a.n_items) {
                const RItem ni = a.items[it + ncl];
                if (ni.kind == ITEM_STAGED) pre = staged_slice_of(a, ni, c, isz, nx);
                else prefetch_next(a, ni, P, c, isz);
            }
            if (!active) continue;
            const float inv = op == OP_SOFTMAX ? 1.0f / st.b : 0.0f;
            for (int k = 0; k < nch; ++k) {
                const long long gb = static_cast<long long>(k) * (kRChunk / 16);
                const long long ge = min(ng, gb + kRChunk / 16);
                for_groups<VW>(buf, gb, ge, tid, T, [&](long long g, const uint4 &w) {
                    float f[V], y[V];
                    decode_group<TIN>(w, f, 1.0f);
                    h_group<V>(op, f, st, inv, y);
                    store_group<TIN, V>(orow + (i_base + g * V) * isz, y, out_vec);
                });
                __syncthreads();  // chunk k of this item is written: its slot takes chunk k of the next
                if (tid == 0 && pre && k < nx.nch) issue_chunk(buf, nx, k, mbar);
            }
            if (tid == 0) pre_issued = pre ? min(nch, nx.nch) : 0;
            for (int e = 0; e < 2; ++e) {  // edge elements, one per thread
                const long long i = e == 0 ? ((own_head && tid < s.h0) ? tid : -1)
                                           : ((own_tail && T - 1 - tid < s.t0) ? s.h0 + s.G * V + (T - 1 - tid) : -1);
                if (i >= 0)
                    store_one<TIN>(orow + i * isz, h_of<TIN>(op, decode_one<TIN>(row + i * isz, 1.0f), st, inv));
            }
        } else {
            // ---- streaming: this CTA's part through the staging buffer as a ring of chunks (many bulk copies in
            // flight), exchange, then the part again (mostly from L2: the cluster read it moments before) and write
            Stream<OP_SOFTMAX> sm;
            Stream<OP_RMS> rs;
            const unsigned char *src = row + s.h0 * isz + s.g_lo * 16;
            const int R = min(a.cap / kRChunk, 14);
            __syncthreads();  // the previous item's reads of buf are done
            // first pass: keep the lines in L2 for the second
            ring_stream(src, ng, buf, R, mbar, phase_bits, a.err, l2_evict_last_policy(),
                        [&](long long, int gn, const unsigned char *cb) {
                for_groups<VW>(cb, 0, gn, tid, T, [&](long long, const uint4 &w) {
                    float f[V];
                    decode_group<TIN>(w, f, 1.0f);
                    if (op == OP_SOFTMAX) sm.add(f);
                    else rs.add(f);
                });
            });
            sweep_edges<TIN>(row, s, P, c, 1.0f, [&](long long, float x) {
                if (op == OP_SOFTMAX) sm.add1(x);
                else rs.add1(x);
            });
            const float2 part = op == OP_SOFTMAX ? block_reduce_stream<OP_SOFTMAX>(sm, red, 0)
                                                 : block_reduce_stream<OP_RMS>(rs, red, 0);
            const Stats st = exchange_sub<TIN>(op, part, slots, xbar, xph, 0, P, c, s, N, a.eps, a.err);
            if (xch) {
                cluster_arrive_release();
                pending = true;
            }
            const float inv = op == OP_SOFTMAX ? 1.0f / st.b : 0.0f;
            ring_stream_again(src, ng, buf, R, mbar, phase_bits, a.err, l2_evict_first_policy(),
                              [&](long long g0, int gn, const unsigned char *cb) {
                for_groups<VW>(cb, 0, gn, tid, T, [&](long long g, const uint4 &w) {
                    float f[V], y[V];
                    decode_group<TIN>(w, f, 1.0f);
                    h_group<V>(op, f, st, inv, y);
                    store_group<TIN, V>(orow + (i_base + (g0 + g) * V) * isz, y, out_vec);
                });
            });
            sweep_edges<TIN>(row, s, P, c, 1.0f, [&](long long i, float x) {
                store_one<TIN>(orow + i * isz, h_of<TIN>(op, x, st, inv));
            });
        }
    }
    if (P > 1) {
        if (pending) cluster_wait_acquire();
        cluster_arrive_release();  // nobody exits while a peer may still push into it
        cluster_wait_acquire();
    }
}

// FP32 and BF16 rows (the ragged entry refuses FP8), vector width 1 or 2 groups.
const void *ragged_kernel(int dt, int vw) {
    if (dt == DT_F32)
        return vw == 2 ? reinterpret_cast<const void *>(&k_ragged<DT_F32, 2>)
                       : reinterpret_cast<const void *>(&k_ragged<DT_F32, 1>);
    return vw == 2 ? reinterpret_cast<const void *>(&k_ragged<DT_BF16, 2>)
                   : reinterpret_cast<const void *>(&k_ragged<DT_BF16, 1>);
}

}  // namespace

struct credit_ragged {
    int device = 0;
    int dtype = 0;
    long long n_rows = 0;
    std::vector<RRow> rows;  // host copy, original order
    const unsigned char *in = nullptr;
    unsigned char *out = nullptr;
    // chosen launch
    int P = 0, threads = 0, cap = 0, clusters = 0, vw = 1;
    long long n_items = 0, n_narrow = 0, n_wide = 0, n_huge = 0;
    RRow *d_rows = nullptr;
    RItem *d_items = nullptr;
    unsigned *d_err = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    float tuned_us = 0.0f;
};

namespace {

// Items for launch shape (P, cap): rows sorted widest first; each row gets
// the smallest power-of-two width w <= P whose slices (plus 32 bytes for an
// unaligned head and tail) fit cap bytes, consecutive rows of one width share
// an item (P / w of them), and rows that fit no width are huge.
void build_items(const std::vector<RRow> &rows, int isz, int P, int cap, std::vector<RItem> &items,
                 std::vector<RRow> &sorted, long long &nn, long long &nw, long long &nh) {
    sorted = rows;
    std::stable_sort(sorted.begin(), sorted.end(), [](const RRow &x, const RRow &y) { return x.cols > y.cols; });
    items.clear();
    nn = nw = nh = 0;
    auto width_of = [&](const RRow &r) -> int {
        const long long groups = r.cols * isz / 16 + 1;
        for (int w = 1; w <= P; w *= 2)
            if ((groups + w - 1) / w * 16 + 32 <= cap) return w;
        return 0;
    };
    size_t i = 0;
    while (i < sorted.size()) {
        const int w = width_of(sorted[i]);
        if (w == 0) {
            items.push_back(RItem{ITEM_HUGE, 1, static_cast<long long>(i), P, 0});
            ++nh;
            ++i;
            continue;
        }
        RItem it{ITEM_STAGED, 0, static_cast<long long>(i), w, 0};
        while (i < sorted.size() && it.count < P / w && width_of(sorted[i]) == w) {
            ++it.count;
            ++i;
        }
        items.push_back(it);
        ++(w == 1 ? nn : nw);
    }
}

credit_status upload_and_launch_config(credit_ragged *h, int P, int threads, int cap, int vw, bool capture,
                                       float *us_out) {
    const int isz = dtype_size(h->dtype);
    const DeviceInfo *di = device_info(h->device);
    std::vector<RItem> items;
    std::vector<RRow> sorted;
    long long nn, nw, nh;
    build_items(h->rows, isz, P, cap, items, sorted, nn, nw, nh);
    const long long smem = kRCtrl + cap;
    if (smem > di->smem_optin) return CREDIT_ERR_UNSUPPORTED;
    const void *fn = ragged_kernel(h->dtype, vw);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(di->smem_optin));
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int maxc = 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(P * 64);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = static_cast<size_t>(smem);
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&maxc, fn, &cfg) != cudaSuccess || maxc <= 0) {
        (void)cudaGetLastError();
        return CREDIT_ERR_UNSUPPORTED;
    }
    const long long ncl = std::min<long long>(maxc, static_cast<long long>(items.size()));
    if (cudaMemcpy(h->d_rows, sorted.data(), sorted.size() * sizeof(RRow), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_items, items.data(), items.size() * sizeof(RItem), cudaMemcpyHostToDevice) != cudaSuccess)
        return CREDIT_ERR_CUDA;
    RaggedArgs ra;
    ra.in = h->in;
    ra.out = h->out;
    ra.rows = h->d_rows;
    ra.items = h->d_items;
    ra.n_items = static_cast<long long>(items.size());
    ra.cap = cap;
    ra.eps = 1e-6f;
    ra.err = h->d_err;
    void *args[] = {&ra};
    cfg.gridDim = dim3(static_cast<unsigned>(P * std::max<long long>(ncl, 1)));
    cfg.stream = h->cap_stream;
    if (capture) {
        if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return CREDIT_ERR_CUDA;
        cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) return CREDIT_ERR_CUDA;
        if (h->exec) cudaGraphExecDestroy(h->exec);
        if (h->graph) cudaGraphDestroy(h->graph);
        h->graph = g;
        if (cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) return CREDIT_ERR_CUDA;
        h->P = P;
        h->vw = vw;
        h->threads = threads;
        h->cap = cap;
        h->clusters = static_cast<int>(ncl);
        h->n_items = static_cast<long long>(items.size());
        h->n_narrow = nn;
        h->n_wide = nw;
        h->n_huge = nh;
        return CREDIT_OK;
    }
    // timing run (median of 3 after a warm-up)
    cudaEvent_t a0, a1;
    cudaEventCreate(&a0);
    cudaEventCreate(&a1);
    std::vector<float> t;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        cudaEventRecord(a0, h->cap_stream);
        e = cudaLaunchKernelExC(&cfg, fn, args);
        cudaEventRecord(a1, h->cap_stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(a1);
        float ms = 0;
        cudaEventElapsedTime(&ms, a0, a1);
        if (k) t.push_back(ms * 1e3f);
    }
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    std::sort(t.begin(), t.end());
    *us_out = t[t.size() / 2];
    return CREDIT_OK;
}

}  // namespace

extern "C" {

credit_status credit_ragged_create(const credit_ragged_row *host_rows, int64_t n, credit_dtype dtype,
                                   const void *in_base, void *out_base, int32_t tune, credit_ragged **out) {
    if (!host_rows || n <= 0 || !in_base || !out_base || !out || dtype < 0 || dtype > 2) return CREDIT_ERR_INVALID_ARG;
    const int isz = dtype_size(dtype);
    if (reinterpret_cast<uintptr_t>(in_base) % isz || reinterpret_cast<uintptr_t>(out_base) % isz)
        return CREDIT_ERR_INVALID_ARG;
    if (dtype == CREDIT_FP8_E4M3) return CREDIT_ERR_UNSUPPORTED;  // ragged FP8 would need per-row scales
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    credit_ragged *h = new (std::nothrow) credit_ragged();
    if (!h) return CREDIT_ERR_INVALID_ARG;
    h->device = dev;
    h->dtype = dtype;
    h->n_rows = n;
    h->in = static_cast<const unsigned char *>(in_base);
    h->out = static_cast<unsigned char *>(out_base);
    h->rows.resize(n);
    for (int64_t i = 0; i < n; ++i) {
        const credit_ragged_row &r = host_rows[i];
        if (r.cols <= 0 || r.in_off < 0 || r.out_off < 0 || (r.op != CREDIT_OP_SOFTMAX && r.op != CREDIT_OP_RMSNORM)) {
            delete h;
            return CREDIT_ERR_INVALID_ARG;
        }
        h->rows[i] = RRow{r.in_off, r.out_off, r.cols, r.op, 0};
    }
    const bool ok = cudaMalloc(&h->d_rows, n * sizeof(RRow)) == cudaSuccess &&
                    cudaMalloc(&h->d_items, n * sizeof(RItem)) == cudaSuccess &&
                    cudaMalloc(&h->d_err, 16) == cudaSuccess &&
                    cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        credit_ragged_destroy(h);
        return CREDIT_ERR_CUDA;
    }
    cudaMemset(h->d_err, 0, 16);
    // autotune: cluster size x staging capacity x threads x vector width, timed on this batch
    const int Ps[3] = {4, 8, 16};
    const int vws[2] = {1, 2};  // 16-byte groups each thread reads before using them
    const int caps[4] = {3 * kRChunk, 4 * kRChunk, 6 * kRChunk, 13 * kRChunk};  // 4, 3, 2, 1 CTAs per SM
    const int thr[2] = {128, 256};  // the kernel is built for up to 256 threads, 4 CTAs per SM (64 registers)
    float best = 1e30f;
    int bP = 16, bcap = caps[3], bthr = 256, bvw = 1;
    if (!tune) {  // fixed launch shape (CREDIT_RAGGED_P / _CHUNKS / _THREADS / _VW override the defaults)
        const char *eP = std::getenv("CREDIT_RAGGED_P"), *eC = std::getenv("CREDIT_RAGGED_CHUNKS");
        const char *eT = std::getenv("CREDIT_RAGGED_THREADS"), *eV = std::getenv("CREDIT_RAGGED_VW");
        if (eP) bP = std::atoi(eP);
        if (eC) bcap = std::atoi(eC) * kRChunk;
        if (eT) bthr = std::atoi(eT);
        if (eV) bvw = std::atoi(eV);
        if (bP < 1 || bP > 16 || bcap < kRChunk || bcap > 13 * kRChunk || bthr < 64 || bthr > 256 || bthr % 32 ||
            (bvw != 1 && bvw != 2)) {
            credit_ragged_destroy(h);
            return CREDIT_ERR_INVALID_ARG;
        }
    } else {
        for (int P : Ps)
            for (int cap : caps)
                for (int t : thr)
                    for (int vw : vws) {
                        float us = 0;
                        if (upload_and_launch_config(h, P, t, cap, vw, false, &us) == CREDIT_OK && us < best) {
                            best = us;
                            bP = P;
                            bcap = cap;
                            bthr = t;
                            bvw = vw;
                        }
                    }
        if (best >= 1e30f) {
            credit_ragged_destroy(h);
            return CREDIT_ERR_UNSUPPORTED;
        }
    }
    h->tuned_us = tune ? best : 0.0f;
    st = upload_and_launch_config(h, bP, bthr, bcap, bvw, true, nullptr);
    if (st != CREDIT_OK) {
        credit_ragged_destroy(h);
        return st;
    }
    cudaStreamSynchronize(h->cap_stream);
    *out = h;
    return CREDIT_OK;
}

credit_status credit_ragged_run(credit_ragged *h, cudaStream_t stream) {
    if (!h || !h->exec) return CREDIT_ERR_INVALID_ARG;
    if (cudaGraphLaunch(h->exec, stream) != cudaSuccess) return CREDIT_ERR_CUDA;
    g_launch_count.fetch_add(1);
    return CREDIT_OK;
}

credit_status credit_ragged_info(const credit_ragged *h, credit_ragged_info_t *out) {
    if (!h || !out) return CREDIT_ERR_INVALID_ARG;
    out->cluster_size = h->P;
    out->threads = h->threads;
    out->staging_bytes = h->cap;
    out->clusters = h->clusters;
    out->items = h->n_items;
    out->narrow_items = h->n_narrow;
    out->wide_items = h->n_wide;
    out->huge_items = h->n_huge;
    out->tuned_us = h->tuned_us;
    out->vector_groups = h->vw;
    return CREDIT_OK;
}

void credit_ragged_destroy(credit_ragged *h) {
    if (!h) return;
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    cudaFree(h->d_rows);
    cudaFree(h->d_items);
    cudaFree(h->d_err);
    delete h;
}

}  // extern "C"
