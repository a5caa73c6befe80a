// credit_prim.cuh -- sm_103a device primitives used by the row kernels.
//
// Inline-PTX wrappers for the pieces of the cluster protocol (CREDIT
// Sec. III-C): bulk-async global->shared copies completed on an mbarrier
// (each CTA stages only its own slice, never a multicast), DSMEM address
// mapping (mapa) and remote stores (st.shared::cluster), and the split
// cluster barrier (barrier.cluster.arrive / wait).  Every spin on an mbarrier
// is bounded by a wall-clock limit; a wait that gives up sets a bit in the
// caller-supplied device error word and returns, so a fault never hangs the
// GPU.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace credit {

enum DType : int { DT_F32 = 0, DT_BF16 = 1, DT_E4M3 = 2, DT_I8 = 3 /* output codes of OP_Q8 only */ };
enum Op : int { OP_SOFTMAX = 0, OP_LSE = 1, OP_LN = 2, OP_RMS = 3, OP_Q8 = 11 /* row-wise int8 quantisation */ };

// Error-word bits (read back by credit_device_error).
enum : unsigned { ERR_TMA_TIMEOUT = 1u, ERR_BAD_LAUNCH = 2u };

// Wall-clock limit of any bounded wait, in nanoseconds (2 s).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ------------------------------------------------------------ mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of `bar`.  Returns false (and flags the
// error word) if the phase did not complete within limit_ns (default 2 s).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned *err,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_timer_ns() - t0 > limit_ns) {
            if (err) atomicOr(err, ERR_TMA_TIMEOUT);
            return false;
        }
    }
}
// The same wait with acquire semantics at cluster scope: for mbarriers that
// peers complete with st.async (the exchange), so that the pushed partials
// are read after the pushes that completed the phase.
__device__ __forceinline__ bool mbar_wait_bounded_cluster(uint64_t *bar, uint32_t parity, unsigned *err) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if ((it & 255u) == 0 && global_timer_ns() - t0 > kWaitLimitNs) {
            if (err) atomicOr(err, ERR_TMA_TIMEOUT);
            return false;
        }
    }
}

// ------------------------------------------------------------ bulk async copy
// Global -> this CTA's shared memory, completion counted in bytes on `bar`.
// dst and src must be 16-byte aligned and bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// L2 eviction policies for cache-hinted copies: keep (data read again soon)
// or evict first (data read once).
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// bulk_g2s with an L2 cache policy for the lines it reads.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                              uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

// Start moving [src, src + bytes) from HBM into L2 (16-byte aligned start, a
// multiple of 16 bytes); no completion to wait for.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// ------------------------------------------------------------ cluster / DSMEM
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// Address of the same shared-memory offset inside CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v2f32(uint32_t addr, float a, float b) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}
// Remote store into a peer CTA's shared memory that completes `bytes` on the
// peer's mbarrier (both addresses already mapped with mapa).
__device__ __forceinline__ void st_async_v2f32(uint32_t addr, float a, float b, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "f"(a), "f"(b), "r"(remote_bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f32(uint32_t addr, float a, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(a),
                 "r"(remote_bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_v4f32(uint32_t addr, const float4 &v, uint32_t remote_bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                     addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(remote_bar)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
// Release fence at cluster scope restricted to this CTA's shared memory: the
// thread's earlier shared::cta accesses (and those ordered before them by
// CTA-scope synchronisation) become ordered before its later release patterns
// at cluster scope -- here, before the st.async that pushes a partial into a
// peer, which is what keeps a peer's next push from overtaking this CTA's
// reads of its own exchange slots.  Far cheaper than fence.acq_rel.cluster,
// which also drains global-memory operations.
__device__ __forceinline__ void fence_release_smem_cluster() {
    asm volatile("fence.release.sync_restrict::shared::cta.cluster;" ::: "memory");
}
// Named barrier over the first `nthreads` threads (a multiple of 32).
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Split cluster barrier.  All threads of every CTA execute these.
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive_release() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ------------------------------------------------------------ tensor memory
// tcgen05 allocation and 32-bit-column loads / stores (sm_100-family).  A
// warp reaches only its lane quarter: lanes 32 * (warp % 4) .. + 31; with the
// 32x32b shape thread t of the warp reads / writes lane 32 * (warp % 4) + t,
// one 32-bit column per register, at consecutive columns.  The load waits for
// its own completion inside the same asm statement, so the compiler never
// sees its registers before the data is there.
__device__ __forceinline__ void tm_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tm_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// r[0..15] <- 16 consecutive columns of this thread's lane
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
                 "tcgen05.wait::ld.sync.aligned;"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
}

// Issue-only store.  tcgen05.st reads its source registers when it issues;
// tm_wait_st() then waits for every store this thread issued (before the
// TMEM words are handed to another warp).
__device__ __forceinline__ void tm_st16_issue(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
                 "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------------------------ math
// 2^x on the SFU (ex2.approx, subnormal results kept).  exp(x) = 2^(x*log2 e).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 2^x on the SFU with subnormal results flushed to zero (ex2.approx.ftz: the
// bare SFU op).  For terms of a softmax sum whose largest term is 1: a flushed
// term is below 2^-126, so N of them move the sum by less than N 2^-126.
__device__ __forceinline__ float ex2_ftz(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 2^x for two halves at once (ex2.approx.f16x2: relative error about 2^-9.9);
// the FP8 softmax output codes, whose spacing is 2^-3 relative, are decided
// from it.
__device__ __forceinline__ __half2 ex2_h2(__half2 x) {
    uint32_t y;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(*reinterpret_cast<const uint32_t *>(&x)));
    return *reinterpret_cast<const __half2 *>(&y);
}
// Sum of V values (V = 2, 4, 8, 16) as a pairwise tree on packed f32x2 adds.
template <int V>
__device__ __forceinline__ float sum_tree(const float (&e)[V]) {
    if constexpr (V == 1) {
        return e[0];
    } else if constexpr (V == 2) {
        return e[0] + e[1];
    } else {
        float h[V / 2];
#pragma unroll
        for (int j = 0; j < V / 4; ++j) {
            const float2 r = __fadd2_rn(make_float2(e[4 * j], e[4 * j + 1]), make_float2(e[4 * j + 2], e[4 * j + 3]));
            h[2 * j] = r.x;
            h[2 * j + 1] = r.y;
        }
        return sum_tree<V / 2>(h);
    }
}
constexpr float kLog2e = 1.4426950408889634f;
// 1/x on the SFU (rcp.approx: relative error below 2^-22 for normal x; one
// instruction, no special-case branch).  The counts it inverts are positive
// integers below 2^24.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float exp_fast(float x) { return ex2_approx(x * kLog2e); }
// exp(x - m) 2^c as 2^((x - m) log2 e + c): one subtraction, one FMA, one SFU
// op.  The difference x - m is exact for the terms near the maximum m
// (Sterbenz), so the error depends on |x - m| (relative 2^-24 |x - m| log2 e
// ln 2 at most, from rounding the exponent, plus log2 e's own rounding), not on
// |m|: logits of any magnitude keep the FP32 bound.  c is the caller's
// log2-domain scale (-log2 S for a softmax, log2 448 for FP8 codes).
// The power is taken as 2^-24 * ex2.ftz(t + 24): every FP32 result down to the
// smallest subnormal (t >= -149) comes from a normal SFU result, and the
// multiply by 2^-24 is exact for normal results and rounds subnormal ones
// correctly (the bare flush-to-zero SFU op plus one multiply).
constexpr float kExpLift = 24.0f, kExpDrop = 5.9604644775390625e-8f;  // the lift 24 and 2^-24
__device__ __forceinline__ float exp_sub(float x, float m, float c) {
    return ex2_ftz(fmaf(x - m, kLog2e, c + kExpLift)) * kExpDrop;
}
// exp_sub over a group, two elements per packed f32x2 subtraction and FMA.
template <int V>
__device__ __forceinline__ void exp_sub_group(const float (&f)[V], float m, float c, float (&y)[V]) {
    if constexpr (V % 2 == 0) {
#pragma unroll
        for (int j = 0; j < V; j += 2) {
            const float cl = c + kExpLift;
            const float2 t = __ffma2_rn(__fadd2_rn(make_float2(f[j], f[j + 1]), make_float2(-m, -m)),
                                        make_float2(kLog2e, kLog2e), make_float2(cl, cl));
            const float2 e = __fmul2_rn(make_float2(ex2_ftz(t.x), ex2_ftz(t.y)), make_float2(kExpDrop, kExpDrop));
            y[j] = e.x;
            y[j + 1] = e.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) y[j] = exp_sub(f[j], m, c);
    }
}

// ------------------------------------------------------------ element formats
template <int DT> struct Fmt;
template <> struct Fmt<DT_F32> {
    static constexpr int size = 4;
    static constexpr int V = 4;   // elements per 16-byte group
};
template <> struct Fmt<DT_BF16> {
    static constexpr int size = 2;
    static constexpr int V = 8;
};
template <> struct Fmt<DT_E4M3> {
    static constexpr int size = 1;
    static constexpr int V = 16;
};
template <> struct Fmt<DT_I8> {
    static constexpr int size = 1;
    static constexpr int V = 16;
};

// Row-wise int8 codes.  With the row scale s = fl(amax / 127) and inv = the
// correctly rounded 1 / s, the code of x is rint(fl(x / s)) (ties to even),
// clamped to +-127.  The codes are carried as "biased" floats u = code +
// kQ8Bias: for an integer |k| < 2^22 the bits of k + 1.5 * 2^23 are
// 0x4B400000 + k, so the low byte of u's bits is k's two's-complement byte
// (the packing below reads it directly).  Fast path: t = x * inv is within
// 3 * 2^-24 * 128 < 2^-15 of fl(x / s) (three roundings of relative size
// <= 2^-24, |x / s| <= 127.00001 when s is normal), so t + kQ8Bias, rounded
// to the nearest integer with ties to even, carries the same code unless t
// lies within 2^-14 of a half-integer; |rint(t)| <= 127 needs no clamp.  Near
// a half-integer, for a non-finite t, or for a subnormal s (whose rounding
// can push x / s past 127.5), the exact quotient decides, clamped.
constexpr float kQ8Bias = 12582912.0f;  // 1.5 * 2^23
__device__ __forceinline__ float q8_exact(float x, float s) {
    return fminf(fmaxf(rintf(__fdiv_rn(x, s)), -127.0f), 127.0f) + kQ8Bias;
}
__device__ __forceinline__ bool q8_near(float t, float u) {
    return !(fabsf(fabsf(t - (u - kQ8Bias)) - 0.5f) >= 0x1p-14f);
}
__device__ __forceinline__ float q8_code(float x, float s, float inv) {
    const float t = x * inv;
    const float u = t + kQ8Bias;
    return (q8_near(t, u) || !(s >= 0x1p-126f)) ? q8_exact(x, s) : u;
}
// The same for N elements with one branch: if any of them needs the exact
// quotient, all N take it.
template <int N>
__device__ __forceinline__ void q8_codes(const float (&x)[N], float s, float inv, float (&y)[N]) {
    bool near = !(s >= 0x1p-126f);
#pragma unroll
    for (int q = 0; q < N; ++q) {
        const float t = x[q] * inv;
        y[q] = t + kQ8Bias;
        near |= q8_near(t, y[q]);
    }
    if (near) {
#pragma unroll
        for (int q = 0; q < N; ++q) y[q] = q8_exact(x[q], s);
    }
}

// Decode one 16-byte group (already loaded as uint4) into floats.
template <int DT>
__device__ __forceinline__ void decode_group(const uint4 &w, float (&f)[Fmt<DT>::V], float scale) {
    if constexpr (DT == DT_F32) {
        f[0] = __uint_as_float(w.x);
        f[1] = __uint_as_float(w.y);
        f[2] = __uint_as_float(w.z);
        f[3] = __uint_as_float(w.w);
    } else if constexpr (DT == DT_BF16) {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            f[2 * k] = __uint_as_float(u[k] << 16);
            f[2 * k + 1] = __uint_as_float(u[k] & 0xFFFF0000u);
        }
    } else {
        const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __nv_fp8x2_storage_t pair = static_cast<__nv_fp8x2_storage_t>((u[k] >> (16 * h)) & 0xFFFFu);
                __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2(pair, __NV_E4M3);
                float2 ff = __half22float2(*reinterpret_cast<__half2 *>(&hr));
                f[4 * k + 2 * h] = ff.x * scale;
                f[4 * k + 2 * h + 1] = ff.y * scale;
            }
        }
    }
}

// Decode a single element from raw storage.
template <int DT>
__device__ __forceinline__ float decode_one(const unsigned char *p, float scale) {
    if constexpr (DT == DT_F32) {
        return *reinterpret_cast<const float *>(p);
    } else if constexpr (DT == DT_BF16) {
        return __uint_as_float(static_cast<uint32_t>(*reinterpret_cast<const uint16_t *>(p)) << 16);
    } else {
        __half_raw hr = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(*p), __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&hr)) * scale;
    }
}

// Encode / store one element.
template <int DT>
__device__ __forceinline__ void store_one(unsigned char *p, float v) {
    if constexpr (DT == DT_F32) {
        *reinterpret_cast<float *>(p) = v;
    } else if constexpr (DT == DT_BF16) {
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(p) = b;
    } else if constexpr (DT == DT_I8) {  // v is a biased code (q8_code): its low byte
        *p = static_cast<unsigned char>(__float_as_uint(v) & 0xFFu);
    } else {
        *p = static_cast<unsigned char>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
    }
}

// Pack V floats into the storage bytes of DT (V * size bytes, V*size % 4 == 0).
template <int DT, int V>
__device__ __forceinline__ void pack_words(const float (&y)[V], uint32_t (&w)[(V * Fmt<DT>::size) / 4]) {
    if constexpr (DT == DT_F32) {
#pragma unroll
        for (int k = 0; k < V; ++k) w[k] = __float_as_uint(y[k]);
    } else if constexpr (DT == DT_BF16) {
#pragma unroll
        for (int k = 0; k < V / 2; ++k) {
            __nv_bfloat162 b = __floats2bfloat162_rn(y[2 * k], y[2 * k + 1]);
            w[k] = *reinterpret_cast<uint32_t *>(&b);
        }
    } else if constexpr (DT == DT_I8) {  // y holds biased codes (q8_code): the low byte of each
#pragma unroll
        for (int k = 0; k < V / 4; ++k)
            w[k] = __byte_perm(__byte_perm(__float_as_uint(y[4 * k]), __float_as_uint(y[4 * k + 1]), 0x0040),
                               __byte_perm(__float_as_uint(y[4 * k + 2]), __float_as_uint(y[4 * k + 3]), 0x0040),
                               0x5410);
    } else {
#pragma unroll
        for (int k = 0; k < V / 4; ++k) {
            uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(y[4 * k], y[4 * k + 1]), __NV_SATFINITE, __NV_E4M3);
            uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(y[4 * k + 2], y[4 * k + 3]), __NV_SATFINITE, __NV_E4M3);
            w[k] = (lo & 0xFFFFu) | (hi << 16);
        }
    }
}

// Store V outputs at p.  vec: p is aligned to min(16, V*size) bytes.
template <int DT, int V>
__device__ __forceinline__ void store_group(unsigned char *p, const float (&y)[V], bool vec) {
    constexpr int bytes = V * Fmt<DT>::size;
    if (vec) {
        uint32_t w[bytes / 4];
        pack_words<DT, V>(y, w);
        if constexpr (bytes >= 16) {
#pragma unroll
            for (int k = 0; k < bytes / 16; ++k)
                *reinterpret_cast<uint4 *>(p + 16 * k) = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        } else if constexpr (bytes == 8) {
            *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
        } else {
            *reinterpret_cast<uint32_t *>(p) = w[0];
        }
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) store_one<DT>(p + k * Fmt<DT>::size, y[k]);
    }
}

// ------------------------------------------------------------ global loads
__device__ __forceinline__ uint4 ld_global_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}
// 16-byte load / store with an L2 cache policy (l2_evict_last_policy, ...).
__device__ __forceinline__ uint4 ld_global_v4_hint(const void *p, uint64_t policy) {
    uint4 v;
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(policy));
    return v;
}
__device__ __forceinline__ void st_global_v4_hint(void *p, const uint4 &v, uint64_t policy) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(policy)
                 : "memory");
}
__device__ __forceinline__ uint4 ld_global_stream_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// ------------------------------------------------------------ warp/block reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Deterministic block all-reduce (sum or max) through `red` (>= 33 floats).
// Every thread returns the same value.  Contains two __syncthreads.
template <bool MAX>
__device__ __forceinline__ float block_allreduce(float v, float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = MAX ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        float t = lane < nw ? red[lane] : (MAX ? -INFINITY : 0.0f);
        t = MAX ? warp_max(t) : warp_sum(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

}  // namespace credit
