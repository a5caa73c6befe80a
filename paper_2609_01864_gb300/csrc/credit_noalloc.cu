// credit_noalloc.cu -- split-row two-pass path with file-scope scratch.
//
// credit_run_two_pass_noalloc() runs the same two kernels as the split-row
// two-pass path of credit_run_ex() (a statistics sweep writing per-CTA
// partials, then a sweep that combines them and writes the output), but it
// keeps the partials in the fixed-size device array below instead of the
// workspace that credit_init() allocates.  It exists for callers that cannot
// allocate device memory: a framework whose caching allocator owns the device
// heap and hands a library only finished buffers (a cudaMalloc behind its
// back would fragment that heap or fail once the allocator has reserved it),
// or an embedding that forbids allocation after start-up.  Nothing in this
// file allocates.
#include <cuda.h>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_rows.cuh"

namespace credit {
bool kernels_tin0(int op, int tout, KernelSet *ks);
bool kernels_tin1(int op, int tout, KernelSet *ks);
bool kernels_tin2(int op, int tout, KernelSet *ks);
extern std::atomic<long long> g_launch_count;
}  // namespace credit

using namespace credit;

namespace {

// 4 MiB of partials: 4 floats per (row, CTA) pair, so one launch covers at
// most kStaticPairs (row, CTA) pairs; larger calls are split into launches.
constexpr long long kStaticFloats = 1LL << 20;
constexpr long long kStaticPairs = kStaticFloats / 4;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_credit_static_ws[kStaticFloats];

std::mutex g_mu;
float *g_static_ptr[kMaxDevices] = {};
unsigned long long g_static_ctx[kMaxDevices] = {};  // context the address belongs to (0: not looked up)

// Unique ID of the calling thread's current context (0 if it cannot be had).
// The driver entry points come through the runtime, so the library does not
// link libcuda itself.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
        (void)cudaGetLastError();
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr ||
        get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the static scratch on `dev`, looked up with that device
// current: once per device, and again only if the device's context has
// changed since (cudaDeviceReset destroys the context, and the array gets a
// new address when the module is loaded into the next one).  nullptr if the
// lookup fails.  The caller has made `dev` current and initialised its
// context (cudaSetDevice / a first runtime call).
float *static_scratch(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    const unsigned long long ctx = current_context_id();
    if (g_static_ptr[dev] == nullptr || ctx == 0 || ctx != g_static_ctx[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_credit_static_ws) != cudaSuccess || p == nullptr) {
            (void)cudaGetLastError();
            g_static_ptr[dev] = nullptr;
            g_static_ctx[dev] = 0;
            return nullptr;
        }
        g_static_ptr[dev] = static_cast<float *>(p);
        g_static_ctx[dev] = ctx;
    }
    return g_static_ptr[dev];
}

cudaError_t launch_plain(const void *fn, unsigned grid, unsigned block, cudaStream_t s, void **args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = s;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

extern "C" credit_status credit_run_two_pass_noalloc(const credit_args *a, int32_t ctas_per_row,
                                                     cudaStream_t stream) {
    credit_status st = validate_args(a);
    if (st != CREDIT_OK) return st;
    if (a->rows == 0) return CREDIT_OK;
    if (ctas_per_row < 2 || ctas_per_row > 4096) return CREDIT_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CREDIT_ERR_CUDA;
    float *ws = static_scratch(dev);
    if (ws == nullptr) return CREDIT_ERR_CUDA;

    const int tin = a->in_dtype;
    const bool lse = a->op == OP_LSE;
    const int tout = lse ? DT_F32 : a->out_dtype;
    KernelSet ks{};
    const bool ok = tin == DT_F32 ? kernels_tin0(a->op, tout, &ks)
                    : tin == DT_BF16 ? kernels_tin1(a->op, tout, &ks)
                                     : kernels_tin2(a->op, tout, &ks);
    if (!ok) return CREDIT_ERR_UNSUPPORTED;

    const int isz = dtype_size(tin), osz = dtype_size(tout);
    const int G = ctas_per_row;
    const long long rows_per_launch = kStaticPairs / G;
    const bool fp8_stage = (a->op == OP_LN || a->op == OP_RMS) && tout == DT_E4M3;
    // the split two-pass path's default CTA size (credit_run_ex with threads = 0): the partials are then
    // formed over the same thread slices and merged in the same order, so both entries agree bit for bit
    const unsigned threads = isz <= 2 ? 256 : 512;

    RowArgs base{};
    base.in = static_cast<const unsigned char *>(a->in);
    base.out = static_cast<unsigned char *>(a->out);
    base.cols = a->cols;
    base.ld_in = a->ld_in ? a->ld_in : a->cols;
    base.ld_out = a->ld_out ? a->ld_out : a->cols;
    base.in_scale = a->in_scale;
    base.out_scale = a->out_scale;
    base.gamma = a->gamma;
    base.beta = a->beta;
    base.eps = a->eps < 0.0f ? (a->op == OP_RMS ? 1e-6f : 1e-5f) : a->eps;
    base.err = nullptr;  // the two-pass kernels never wait on anything
    base.ws = ws;
    base.G = G;

    for (long long r0 = 0; r0 < a->rows; r0 += rows_per_launch) {
        const long long n = a->rows - r0 < rows_per_launch ? a->rows - r0 : rows_per_launch;
        RowArgs r = base;
        r.in = base.in + r0 * base.ld_in * isz;
        r.out = lse ? base.out + r0 * 4 : base.out + r0 * base.ld_out * osz;
        if (base.in_scale) r.in_scale = base.in_scale + r0;
        if (base.out_scale) r.out_scale = base.out_scale + r0;
        r.rows = n;
        void *args[] = {&r};
        const unsigned grid = static_cast<unsigned>(G * n);
        cudaError_t e = launch_plain(ks.tp_stats, grid, threads, stream, args);
        if (e != cudaSuccess) return CREDIT_ERR_CUDA;
        g_launch_count.fetch_add(1);
        if (lse) {
            long long nn = n;
            void *args2[] = {&r, &nn};
            e = launch_plain(ks.tp_lse_final, static_cast<unsigned>((n + 255) / 256), 256, stream, args2);
            if (e != cudaSuccess) return CREDIT_ERR_CUDA;
            g_launch_count.fetch_add(1);
            continue;
        }
        if (fp8_stage) {
            e = launch_plain(ks.tp_amax, grid, threads, stream, args);
            if (e != cudaSuccess) return CREDIT_ERR_CUDA;
            g_launch_count.fetch_add(1);
        }
        e = launch_plain(ks.tp_apply, grid, threads, stream, args);
        if (e != cudaSuccess) return CREDIT_ERR_CUDA;
        g_launch_count.fetch_add(1);
    }
    return CREDIT_OK;
}
