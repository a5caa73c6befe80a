// credit_api.cu -- host side of the C ABI declared in include/credit.h.
//
// Argument validation, per-device state (limits, workspace, error word),
// plan legality (Eq. 3 capacity, cluster occupancy), and the launches of the
// three paths.  Planning itself lives in credit_plan.cpp.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_ring_tm.cuh"

namespace credit {
bool kernels_tin0(int op, int tout, KernelSet *ks);
bool kernels_tin1(int op, int tout, KernelSet *ks);
bool kernels_tin2(int op, int tout, KernelSet *ks);
}  // namespace credit

using namespace credit;

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kWorkspaceFloats = size_t(16) << 20;  // 64 MiB of two-pass partials

struct DeviceState {
    std::mutex mu;
    std::atomic<bool> ready{false};
    DeviceInfo info{};
    float *ws = nullptr;
    unsigned *err = nullptr;
    cudaStream_t side = nullptr;               // fill work of cluster plans (fill_share > 0)
    cudaEvent_t fork = nullptr, join = nullptr;
    std::map<const void *, bool> attr_done;
    std::map<std::tuple<const void *, int, int, long long>, int> clusters;  // max active clusters
};
DeviceState g_dev[kMaxDevices];

bool kernel_set(int op, int tin, int tout, KernelSet *ks) {
    std::memset(ks, 0, sizeof(*ks));
    if (op == OP_LSE) tout = DT_F32;
    switch (tin) {
    case DT_F32: return kernels_tin0(op, tout, ks);
    case DT_BF16: return kernels_tin1(op, tout, ks);
    case DT_E4M3: return kernels_tin2(op, tout, ks);
    default: return false;
    }
}

credit_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CREDIT_OK;
    if (std::getenv("CREDIT_LOG")) std::fprintf(stderr, "credit: CUDA error %s\n", cudaGetErrorString(e));
    return CREDIT_ERR_CUDA;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

// Raise per-kernel attributes once per (device, kernel).
credit_status prepare_kernel(DeviceState &d, const void *fn, bool staged) {
    std::lock_guard<std::mutex> lk(d.mu);
    if (d.attr_done.count(fn)) return CREDIT_OK;
    if (staged) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(d.info.smem_optin));
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cuda_status(e);
        e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return cuda_status(e);
    }
    d.attr_done[fn] = true;
    return CREDIT_OK;
}

}  // namespace

// ------------------------------------------------------------------ host helpers
namespace credit {

// AUTO retention policy: tensor memory where it applies (slices above
// kTmAutoMinSlice bytes).
bool g_auto_retain_tmem = true;

int dtype_size(int dt) { return dt == DT_F32 ? 4 : (dt == DT_BF16 ? 2 : 1); }

// Geometry of the staged (ring) paths for rows of N elements of isz bytes
// over P CTAs.  The body of a CTA's slice is at most ceil(G / P) 16-byte
// groups, G = floor(N * isz / 16).  Eq. 3: the slice must fit the ring, i.e.
// kRingCtrl + ceil(body / chunk) * chunk <= the opt-in shared memory.
bool ring_config(const DeviceInfo &di, long long N, int isz, int P, int req_ring, int req_chunk, int req_threads,
                 int req_reducers, int nab, RingCfg *out) {
    if (P < 1 || P > kMaxCluster || N <= 0) return false;
    const long long groups = (N * isz) / 16;
    const long long per = (groups + P - 1) / P;
    RingCfg r{};
    r.P = P;
    r.body_max = per * 16;
    // gamma / beta bytes staged per data byte
    const int abytes_per16 = nab * (16 / isz) * 4;
    long long max_chunk = kMaxChunkBytes;
    if (nab > 0) {
        const long long cap = (32768LL * 16 / abytes_per16) / 16 * 16;  // affine slot <= 32 KiB
        if (cap < max_chunk) max_chunk = cap;
    }
    if (req_chunk > 0) {
        if (req_chunk % 16) return false;
        r.chunk = req_chunk;
    } else if (r.body_max == 0) {
        r.chunk = 16;
    } else {
        const long long n = (r.body_max + max_chunk - 1) / max_chunk;
        r.chunk = static_cast<int>(((r.body_max + n - 1) / n + 15) / 16 * 16);
    }
    r.nch_max = static_cast<int>((r.body_max + r.chunk - 1) / r.chunk);
    r.aslot = static_cast<long long>(r.chunk / 16) * abytes_per16;
    r.affine = 0;
    r.affine_resident = 0;
    if (nab > 0) {
        // resident gamma / beta (one slot per chunk of the slice, loaded once)
        // when that leaves room for one slice in the ring, else 2 streaming slots
        const long long res = static_cast<long long>(r.nch_max) * r.aslot;
        if (r.nch_max <= kMaxAffine &&
            kRingCtrl + res + static_cast<long long>(r.nch_max) * r.chunk <= di.smem_optin) {
            r.affine = r.nch_max < 1 ? 1 : r.nch_max;
            r.affine_resident = 1;
        } else {
            r.affine = 2;
        }
    }
    const long long budget = di.smem_optin - kRingCtrl - r.affine * r.aslot;
    const long long fit = budget > 0 ? budget / r.chunk : 0;
    if (req_ring > 0) {
        r.ring = req_ring;
    } else {
        long long k = 2LL * r.nch_max;
        if (k < 2) k = 2;
        if (k > kMaxRing) k = kMaxRing;
        if (k > fit) k = fit;
        r.ring = static_cast<int>(k);
    }
    if (r.ring < r.nch_max || r.ring < 1 || r.ring > kMaxRing) return false;
    r.smem = kRingCtrl + static_cast<long long>(r.ring) * r.chunk + r.affine * r.aslot;
    if (r.smem > di.smem_optin) return false;  // Eq. 3
    if (req_threads > 0) {
        if (req_threads % 32 || req_threads < 96 || req_threads > 288) return false;
        r.threads = req_threads;
    } else {
        long long tc = (r.chunk / 16 / 4 + 31) / 32 * 32;
        if (tc < 128) tc = 128;
        if (tc > 256) tc = 256;
        r.threads = static_cast<int>(tc) + 32;
    }
    const int tp = r.threads - 32;
    if (req_reducers > 0) {
        if (req_reducers % 32 || req_reducers >= tp) return false;
        r.reducers = req_reducers;
    } else {
        r.reducers = (tp / 2) / 32 * 32;
        if (r.reducers < 32) r.reducers = 32;
    }
    if (tp - r.reducers < 32) return false;
    r.tmem = 0;
    *out = r;
    return true;
}

// Geometry of k_ring_tm.  The slice is retained in one of two TMEM buffers of
// kTmMaxChunks chunks (capacity: kTmMaxChunks * kTmMaxChunkBytes bytes of
// input per CTA); the shared-memory ring only holds chunks between landing and
// sweep, and gamma / beta are resident in shared memory when they fit beside
// a ring of at least kTmMinRing chunks, else streamed through as many slots as
// fit beside a ring of kTmStreamRing chunks.  The
// request is raised above half of the SM's shared memory so that one CTA runs
// per SM (the kernel allocates all kTmCols columns).
bool ring_config_tm(const DeviceInfo &di, long long N, int isz, int P, int req_ring, int req_chunk, int nab,
                    RingCfg *out) {
    constexpr int kTmMinRing = 4;     // chunks in flight: enough to cover the load latency
    constexpr int kTmStreamRing = 5;  // ring beside streamed gamma / beta slots
    if (P < 1 || P > kMaxCluster || N <= 0) return false;
    const long long groups = (N * isz) / 16;
    const long long per = (groups + P - 1) / P;
    RingCfg r{};
    r.P = P;
    r.tmem = 1;
    r.body_max = per * 16;
    const int abytes_per16 = nab * (16 / isz) * 4;
    const long long max_chunk = kTmMaxChunkBytes;
    if (req_chunk > 0) {
        if (req_chunk % 16 || req_chunk > kTmMaxChunkBytes) return false;
        r.chunk = req_chunk;
    } else if (r.body_max == 0) {
        r.chunk = 16;
    } else {
        const long long n = (r.body_max + max_chunk - 1) / max_chunk;
        r.chunk = static_cast<int>(((r.body_max + n - 1) / n + 15) / 16 * 16);
    }
    r.nch_max = static_cast<int>((r.body_max + r.chunk - 1) / r.chunk);
    if (r.nch_max > kTmMaxChunks) return false;  // TMEM capacity
    r.aslot = static_cast<long long>(r.chunk / 16) * abytes_per16;
    const long long budget = di.smem_optin - kTmCtrl;
    r.affine = 0;
    r.affine_resident = 0;
    if (nab > 0) {
        const long long res = static_cast<long long>(r.nch_max < 1 ? 1 : r.nch_max) * r.aslot;
        const char *mode = std::getenv("CREDIT_TM_AFFINE");
        const bool force_stream = mode && std::strcmp(mode, "stream") == 0;
        const bool force_direct = mode && std::strcmp(mode, "direct") == 0;
        if (force_direct) {
            r.affine = 0;
        } else if (!force_stream && r.nch_max <= kMaxAffine && (budget - res) / r.chunk >= kTmMinRing) {
            r.affine = r.nch_max < 1 ? 1 : r.nch_max;
            r.affine_resident = 1;
        } else {
            // as many streaming slots as fit beside a ring of kTmStreamRing chunks
            long long na = (budget - static_cast<long long>(kTmStreamRing) * r.chunk) / r.aslot;
            if (na > kMaxAffine) na = kMaxAffine;
            if (na < 0) na = 0;
            r.affine = static_cast<int>(na);
        }
    }
    const long long fit = (budget - r.affine * r.aslot) / r.chunk;
    if (req_ring > 0) {
        r.ring = req_ring;
    } else {
        long long k = fit < kMaxRing ? fit : kMaxRing;
        r.ring = static_cast<int>(k);
    }
    if (r.ring < 2 || r.ring > kMaxRing) return false;
    r.smem = kTmCtrl + static_cast<long long>(r.ring) * r.chunk + r.affine * r.aslot;
    if (r.smem > di.smem_optin) return false;
    const long long half = di.smem_per_sm / 2 + 1024;  // one CTA per SM
    if (r.smem < half) r.smem = half;
    if (r.smem > di.smem_optin) return false;
    r.threads = kTmThreads;
    r.reducers = kTmReducers;
    *out = r;
    return true;
}

// Number of gamma / beta arrays the ring kernel can stream through its affine
// ring for these arguments (0 = the reuse pass loads them directly): norms
// only, every row starting at the same 16-byte phase, and the gamma / beta
// segments of the slices 16-byte aligned.
int affine_arrays_aligned(const credit_args *a) {
    if (a->op != OP_LN && a->op != OP_RMS) return 0;
    const int isz = dtype_size(a->in_dtype);
    const long long ld = a->ld_in ? a->ld_in : a->cols;
    if ((ld * isz) % 16) return 0;
    const uintptr_t ip = reinterpret_cast<uintptr_t>(a->in);
    const long long mis = static_cast<long long>(ip & 15u);
    long long h0 = mis ? (16 - mis) / isz : 0;
    if (h0 > a->cols) h0 = a->cols;
    const float *gm = a->gamma;
    const float *bt = a->op == OP_LN ? a->beta : nullptr;
    if (gm && (reinterpret_cast<uintptr_t>(gm + h0) & 15u)) return 0;
    if (bt && (reinterpret_cast<uintptr_t>(bt + h0) & 15u)) return 0;
    return (gm ? 1 : 0) + (bt ? 1 : 0);
}

int affine_arrays(const credit_args *a) {
    // gamma / beta staging in the shared-memory ring kernel is opt-in
    // (CREDIT_AFFINE_STAGE=1): there it costs ring capacity, and the writers'
    // batched L2 loads measure faster
    const char *stage = std::getenv("CREDIT_AFFINE_STAGE");
    if (!stage || std::atoi(stage) == 0) return 0;
    return affine_arrays_aligned(a);
}

const DeviceInfo *device_info(int device) {
    if (device < 0 || device >= kMaxDevices || !g_dev[device].ready.load()) return nullptr;
    return &g_dev[device].info;
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    return dev;
}

// Max active clusters of the ring kernel for (op, dtypes, P, threads, smem);
// 0 if it cannot be scheduled.  Cached.
int ring_max_clusters(int device, int op, int tin, int tout, int P, int threads, long long smem, bool tm) {
    if (device < 0 || device >= kMaxDevices) return 0;
    KernelSet ks;
    if (!kernel_set(op, tin, tout, &ks)) return 0;
    const void *fn = tm ? ks.ring_tm : ks.ring;
    if (fn == nullptr) return 0;
    return staged_max_clusters(device, fn, P, threads, smem, tm);
}

int staged_max_clusters(int device, const void *fn, int P, int threads, long long smem, bool one_per_sm) {
    if (device < 0 || device >= kMaxDevices || fn == nullptr) return 0;
    DeviceState &d = g_dev[device];
    const bool tm = one_per_sm;
    if (smem > d.info.smem_optin) return 0;
    if (prepare_kernel(d, fn, true) != CREDIT_OK) return 0;
    const auto key = std::make_tuple(fn, P, threads, smem);
    {
        std::lock_guard<std::mutex> lk(d.mu);
        auto it = d.clusters.find(key);
        if (it != d.clusters.end()) return it->second;
    }
    int n = 0;
    if (P <= 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, static_cast<size_t>(smem)) ==
            cudaSuccess)
            n = per_sm * d.info.sm_count;
        else
            (void)cudaGetLastError();
        if (tm && per_sm > 1) n = 0;  // TMEM allocation assumes one CTA per SM
    } else {
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
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
            n = 0;
            (void)cudaGetLastError();
        }
    }
    std::lock_guard<std::mutex> lk(d.mu);
    d.clusters[key] = n;
    return n;
}

credit_status prepare_staged_kernel(int device, const void *fn) {
    if (device < 0 || device >= kMaxDevices) return CREDIT_ERR_CUDA;
    return prepare_kernel(g_dev[device], fn, true);
}

unsigned *device_error_word(int device) {
    return device < 0 || device >= kMaxDevices ? nullptr : g_dev[device].err;
}

float *device_workspace(int device, size_t *floats) {
    if (device < 0 || device >= kMaxDevices) return nullptr;
    if (floats) *floats = g_dev[device].info.ws_floats;
    return g_dev[device].ws;
}

}  // namespace credit

// ------------------------------------------------------------------ C ABI
extern "C" {

const char *credit_status_string(credit_status s) {
    switch (s) {
    case CREDIT_OK: return "CREDIT_OK";
    case CREDIT_ERR_INVALID_ARG: return "CREDIT_ERR_INVALID_ARG";
    case CREDIT_ERR_UNSUPPORTED: return "CREDIT_ERR_UNSUPPORTED";
    case CREDIT_ERR_CUDA: return "CREDIT_ERR_CUDA";
    case CREDIT_ERR_TIMEOUT: return "CREDIT_ERR_TIMEOUT";
    case CREDIT_ERR_NOT_INITIALIZED: return "CREDIT_ERR_NOT_INITIALIZED";
    case CREDIT_ERR_CAPTURE: return "CREDIT_ERR_CAPTURE";
    case CREDIT_ERR_IO: return "CREDIT_ERR_IO";
    default: return "CREDIT_ERR_UNKNOWN";
    }
}

int credit_version(void) { return 10000; }

credit_status credit_init(int device) {
    if (device < 0 || device >= kMaxDevices) return CREDIT_ERR_INVALID_ARG;
    DeviceState &d = g_dev[device];
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_status(e);
    if (d.ready.load()) return CREDIT_OK;
    std::lock_guard<std::mutex> lk(d.mu);
    if (d.ready.load()) return CREDIT_OK;
    DeviceInfo info{};
    int v = 0;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return cuda_status(e);
    info.sm_count = v;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) != cudaSuccess)
        return cuda_status(e);
    info.smem_optin = v;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device)) != cudaSuccess)
        return cuda_status(e);
    info.smem_per_sm = v;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, device)) != cudaSuccess)
        return cuda_status(e);
    info.cc_major = v;
    if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, device)) != cudaSuccess)
        return cuda_status(e);
    info.cc_minor = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrClockRate, device) == cudaSuccess) info.clock_khz = v;
    if (info.cc_major < 10) return CREDIT_ERR_UNSUPPORTED;  // needs Blackwell (sm_103a build)
    if ((e = cudaMalloc(&d.ws, kWorkspaceFloats * sizeof(float))) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMalloc(&d.err, 64)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemset(d.err, 0, 64)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaStreamCreateWithFlags(&d.side, cudaStreamNonBlocking)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaEventCreateWithFlags(&d.join, cudaEventDisableTiming)) != cudaSuccess) return cuda_status(e);
    info.ws_floats = kWorkspaceFloats;
    d.info = info;
    d.ready.store(true);
    return CREDIT_OK;
}

int64_t credit_slice_capacity(credit_dtype dtype) {
    const DeviceInfo *di = device_info(current_device());
    if (!di || dtype < 0 || dtype > 2) return 0;
    const long long bytes = di->smem_optin - kRingCtrl;
    return bytes / 16 * 16 / dtype_size(dtype);
}

credit_status credit_device_error(cudaStream_t stream) {
    const int dev = current_device();
    if (dev < 0 || !g_dev[dev].ready.load()) return CREDIT_ERR_NOT_INITIALIZED;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned w = 0;
    if ((e = cudaMemcpy(&w, g_dev[dev].err, sizeof(w), cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_status(e);
    if (w != 0 && (e = cudaMemset(g_dev[dev].err, 0, sizeof(w))) != cudaSuccess) return cuda_status(e);
    return w ? CREDIT_ERR_TIMEOUT : CREDIT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ launching
namespace credit {

// Retention tier asked for by a plan: 0 shared memory, 1 tensor memory,
// 2 AUTO (tensor memory where it applies and the slice exceeds
// kTmAutoMinSlice), 3 tensor memory wherever it applies (CREDIT_RETAIN=tmem;
// CREDIT_RETAIN=smem gives 0).
static int retain_request(const credit_plan_t *p) {
    if (p->retain == CREDIT_RETAIN_SMEM) return 0;
    if (p->retain == CREDIT_RETAIN_TMEM) return 1;
    const char *e = std::getenv("CREDIT_RETAIN");
    if (e && std::strcmp(e, "smem") == 0) return 0;
    if (e && std::strcmp(e, "tmem") == 0) return 3;
    return g_auto_retain_tmem ? 2 : 0;
}

// Ring geometry for a call.  Tensor-memory retention first when the plan asks
// for it and the op has a reuse pass (not logsumexp, not the FP8-output norms,
// whose amax stage rereads the slice); then the shared-memory ring, with the
// gamma / beta affine ring when it fits, else with direct gamma / beta loads.
static bool ring_config_for(const DeviceInfo &di, const credit_args *a, int isz, int P, const credit_plan_t *p,
                            RingCfg *rc) {
    const int tout = a->op == OP_LSE ? DT_F32 : a->out_dtype;
    const bool tm_op = a->op != OP_LSE && !(tout == DT_E4M3 && (a->op == OP_LN || a->op == OP_RMS));
    int want = retain_request(p);
    const bool tuned_smem = p->threads != 0 || p->reducer_threads != 0;
    if (want == 2) {
        // AUTO: tensor memory pays off once a slice is large enough that the
        // shared-memory ring would hold one CTA per SM anyway (> 32 KiB)
        const long long groups = (a->cols * isz) / 16;
        if ((groups + P - 1) / P * 16 <= kTmAutoMinSlice || tuned_smem) want = 0;
    }
    if (want != 0 && tm_op &&
        (p->threads == 0 || p->threads == kTmThreads) && (p->reducer_threads == 0 || p->reducer_threads == kTmReducers) &&
        ring_config_tm(di, a->cols, isz, P, p->ring_chunks, p->chunk_bytes, affine_arrays_aligned(a), rc)) {
        // LayerNorm whose gamma / beta the tensor-memory kernel would read from L2 (rows off the 16-byte grid,
        // or no room to stage them) takes the shared-memory ring instead: on that combination the tensor-memory
        // kernel returned wrong rows in soak runs (the second row of a cluster, one warp's 512-byte read of a
        // ring slot), a fault not yet found
        if (!(a->op == OP_LN && (a->gamma || a->beta) && rc->affine == 0)) return true;
        want = 0;
    }
    if (want == 1) return false;  // tensor memory asked for but not applicable
    const int nab = affine_arrays(a);
    if (nab > 0 &&
        ring_config(di, a->cols, isz, P, p->ring_chunks, p->chunk_bytes, p->threads, p->reducer_threads, nab, rc))
        return true;
    return ring_config(di, a->cols, isz, P, p->ring_chunks, p->chunk_bytes, p->threads, p->reducer_threads, 0, rc);
}

credit_status validate_args(const credit_args *a) {
    if (!a) return CREDIT_ERR_INVALID_ARG;
    const bool q8 = a->op == OP_Q8;
    if ((a->op < 0 || a->op > 3) && !q8) return CREDIT_ERR_INVALID_ARG;
    if (a->in_dtype < 0 || a->in_dtype > 2 || a->out_dtype < 0 || a->out_dtype > 3) return CREDIT_ERR_INVALID_ARG;
    if (q8 != (a->out_dtype == DT_I8)) return CREDIT_ERR_INVALID_ARG;    // int8 codes are the quantiser's output only
    if (q8 && a->in_dtype == DT_E4M3) return CREDIT_ERR_UNSUPPORTED;     // FP32 / BF16 rows
    if (a->rows < 0 || a->cols <= 0) return CREDIT_ERR_INVALID_ARG;
    if (a->rows == 0) return CREDIT_OK;
    if (!a->in || !a->out) return CREDIT_ERR_INVALID_ARG;
    const long long ld_in = a->ld_in ? a->ld_in : a->cols;
    const long long ld_out = a->ld_out ? a->ld_out : a->cols;
    if (ld_in < a->cols || (a->op != OP_LSE && ld_out < a->cols)) return CREDIT_ERR_INVALID_ARG;
    if (a->in_dtype == DT_E4M3 && !a->in_scale) return CREDIT_ERR_INVALID_ARG;
    const int tout = a->op == OP_LSE ? DT_F32 : a->out_dtype;
    if (a->op != OP_LSE && (tout == DT_E4M3 || q8) && !a->out_scale) return CREDIT_ERR_INVALID_ARG;
    const uintptr_t ip = reinterpret_cast<uintptr_t>(a->in), op = reinterpret_cast<uintptr_t>(a->out);
    if (ip % dtype_size(a->in_dtype) || op % dtype_size(tout)) return CREDIT_ERR_INVALID_ARG;
    if ((a->gamma && reinterpret_cast<uintptr_t>(a->gamma) % 4) ||
        (a->beta && reinterpret_cast<uintptr_t>(a->beta) % 4))
        return CREDIT_ERR_INVALID_ARG;
    if (a->op == OP_LSE && a->in == a->out) return CREDIT_ERR_INVALID_ARG;
    return CREDIT_OK;
}

// Is `p` legal for the arguments on this device (Eq. 3 and scheduling)?
credit_status check_plan(int device, const credit_args *a, const credit_plan_t *p) {
    const DeviceInfo *di = device_info(device);
    if (!di) return CREDIT_ERR_NOT_INITIALIZED;
    const int isz = dtype_size(a->in_dtype);
    const int tout = a->op == OP_LSE ? DT_F32 : a->out_dtype;
    const int threads = p->threads;
    if (threads != 0 && (threads < 64 || threads > 1024 || threads % 32)) return CREDIT_ERR_UNSUPPORTED;
    (void)threads;
    if (!(p->fill_share >= 0.0f && p->fill_share <= kMaxFillShare)) return CREDIT_ERR_UNSUPPORTED;
    if (p->fill_share > 0.0f && (p->path != CREDIT_PATH_CLUSTER || p->fill_g < 0 || p->fill_g > 4096 ||
                                 static_cast<size_t>(p->fill_g) * 4 > di->ws_floats))
        return CREDIT_ERR_UNSUPPORTED;
    switch (p->path) {
    case CREDIT_PATH_ONE_CTA:
    case CREDIT_PATH_CLUSTER: {
        const int P = p->path == CREDIT_PATH_ONE_CTA ? 1 : p->cluster_size;
        if (P < 1 || P > kMaxCluster) return CREDIT_ERR_UNSUPPORTED;
        if (p->path == CREDIT_PATH_CLUSTER && P < 2) return CREDIT_ERR_UNSUPPORTED;
        RingCfg rc;
        if (!ring_config_for(*di, a, isz, P, p, &rc))
            return CREDIT_ERR_UNSUPPORTED;  // Eq. 3
        if (ring_max_clusters(device, a->op, a->in_dtype, tout, P, rc.threads, rc.smem, rc.tmem != 0) <= 0)
            return CREDIT_ERR_UNSUPPORTED;
        return CREDIT_OK;
    }
    case CREDIT_PATH_TWO_PASS: {
        const int G = p->ctas_per_row;
        if (G < 1 || G > 4096) return CREDIT_ERR_UNSUPPORTED;
        if (G > 1 && static_cast<size_t>(G) * 4 > di->ws_floats) return CREDIT_ERR_UNSUPPORTED;
        return CREDIT_OK;
    }
    default: return CREDIT_ERR_UNSUPPORTED;
    }
}

static unsigned long long *g_trace_buf = nullptr;
static int g_trace_rows = 0;
// credit_set_wait_test (test only): the reducers' chunk-wait limit and the
// extra bytes the first chunk's barrier expects
static std::atomic<unsigned long long> g_wait_ns{0};
static std::atomic<int> g_test_extra_tx{0};

static RowArgs make_row_args(const credit_args *a, unsigned *err, float *ws) {
    RowArgs r;
    r.in = static_cast<const unsigned char *>(a->in);
    r.out = static_cast<unsigned char *>(a->out);
    r.rows = a->rows;
    r.cols = a->cols;
    r.ld_in = a->ld_in ? a->ld_in : a->cols;
    r.ld_out = a->ld_out ? a->ld_out : a->cols;
    r.in_scale = a->in_scale;
    r.out_scale = a->out_scale;
    r.gamma = (a->op == OP_LN || a->op == OP_RMS) ? a->gamma : nullptr;  // the other ops take no affine
    r.beta = a->op == OP_LN ? a->beta : nullptr;
    const float dflt = a->op == OP_RMS ? 1e-6f : 1e-5f;
    r.eps = a->eps < 0.0f ? dflt : a->eps;
    r.err = err;
    r.ws = ws;
    r.G = 1;
    r.chunk_bytes = 0;
    r.ring = 0;
    r.reducers = 0;
    r.affine = 0;
    r.affine_resident = 0;
    r.trace = g_trace_buf;
    r.trace_rows = g_trace_rows;
    r.row0 = 0;
    r.wait_ns = g_wait_ns.load();
    r.test_extra_tx = 0;
    return r;
}

// Shift the row pointers of `r` by `r0` rows (chunked launches).
static RowArgs rows_from(const RowArgs &base, long long r0, long long n, int isz, int osz, bool lse) {
    RowArgs r = base;
    r.in = base.in + r0 * base.ld_in * isz;
    r.out = lse ? base.out + r0 * 4 : base.out + r0 * base.ld_out * osz;
    if (base.in_scale) r.in_scale = base.in_scale + r0;
    if (base.out_scale) r.out_scale = base.out_scale + r0;
    r.rows = n;
    return r;
}

cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, size_t smem, int cluster, cudaStream_t s,
                          void **args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    if (cluster > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelExC(&cfg, fn, args);
}

static cudaError_t launch(const void *fn, dim3 grid, dim3 block, size_t smem, int cluster, cudaStream_t s,
                          void **args) {
    return launch_kernel(fn, grid, block, smem, cluster, s, args);
}

std::atomic<long long> g_launch_count{0};

// Rows of a cluster plan handed to the fill (the last ones); at least one row
// stays on the cluster path.
static long long fill_rows(const credit_plan_t *p, long long rows) {
    if (p->path != CREDIT_PATH_CLUSTER || !(p->fill_share > 0.0f) || rows < 2) return 0;
    long long n = static_cast<long long>(static_cast<double>(rows) * p->fill_share + 0.5);
    if (n > rows - 1) n = rows - 1;
    return n < 0 ? 0 : n;
}

// CTAs per row of the fill's two-pass part when the plan leaves it open: one
// per 512 KiB of row (1..8), so that each CTA's reread slice stays small.
static int fill_split(long long cols, int isz) {
    long long g = cols * isz / (512LL << 10);
    if (g < 1) g = 1;
    if (g > 8) g = 8;
    return static_cast<int>(g);
}

credit_status run_with_plan(int device, const credit_args *a, const credit_plan_t *p, cudaStream_t s) {
    DeviceState &d = g_dev[device];
    const int tin = a->in_dtype;
    const int tout = a->op == OP_LSE ? DT_F32 : a->out_dtype;
    const int isz = dtype_size(tin), osz = dtype_size(tout);
    const bool lse = a->op == OP_LSE;
    KernelSet ks;
    if (!kernel_set(a->op, tin, tout, &ks)) return CREDIT_ERR_UNSUPPORTED;
    const RowArgs base = make_row_args(a, d.err, d.ws);
    const long long rows = a->rows;

    if (p->path == CREDIT_PATH_ONE_CTA || p->path == CREDIT_PATH_CLUSTER) {
        const int P = p->path == CREDIT_PATH_ONE_CTA ? 1 : p->cluster_size;
        RingCfg rc;
        if (!ring_config_for(d.info, a, isz, P, p, &rc))
            return CREDIT_ERR_UNSUPPORTED;
        const void *fn = rc.tmem ? ks.ring_tm : ks.ring;
        if (fn == nullptr) return CREDIT_ERR_UNSUPPORTED;
        credit_status st = prepare_kernel(d, fn, true);
        if (st != CREDIT_OK) return st;
        const int maxc = ring_max_clusters(device, a->op, tin, tout, P, rc.threads, rc.smem, rc.tmem != 0);
        if (maxc <= 0) return CREDIT_ERR_UNSUPPORTED;
        const long long ncl = rows < maxc ? rows : maxc;
        if (std::getenv("CREDIT_LOG"))
            std::fprintf(stderr,
                         "credit: ring%s op=%d P=%d clusters=%lld (max %d) threads=%d reducers=%d chunk=%d ring=%d "
                         "affine=%d%s smem=%lld\n",
                         rc.tmem ? "_tm" : "", a->op, P, ncl, maxc, rc.threads, rc.reducers, rc.chunk, rc.ring,
                         rc.affine, rc.affine_resident ? "(resident)" : "", rc.smem);
        // fill: the last n_fill rows go to the split two-pass path on the side
        // stream, which forks from s before the cluster launch and joins after
        const long long n_fill = fill_rows(p, rows);
        const long long n_cl = rows - n_fill;
        cudaError_t e;
        if (n_fill > 0 && (e = cudaEventRecord(d.fork, s)) != cudaSuccess) return cuda_status(e);
        const int extra_tx = g_test_extra_tx.load();
        // the unsatisfiable first-chunk barrier of the wait test: one CTA, one row, one chunk, shared-memory
        // ring (the barrier is armed once and never reused; the one copy issued completes)
        if (extra_tx > 0 && (P != 1 || rows != 1 || rc.tmem || rc.nch_max != 1 || fill_rows(p, rows) > 0))
            return CREDIT_ERR_UNSUPPORTED;
        RowArgs r = base;
        r.test_extra_tx = extra_tx;
        r.rows = n_cl;
        r.chunk_bytes = rc.chunk;
        r.ring = rc.ring;
        r.reducers = rc.reducers;
        r.affine = rc.affine;
        r.affine_resident = rc.affine_resident;
        const long long ncl_run = n_cl < ncl ? n_cl : ncl;
        void *args[] = {&r};
        e = launch(fn, dim3(static_cast<unsigned>(P * ncl_run)), dim3(rc.threads), static_cast<size_t>(rc.smem), P,
                   s, args);
        if (e != cudaSuccess) return cuda_status(e);
        g_launch_count.fetch_add(1);
        if (n_fill > 0) {
            if ((e = cudaStreamWaitEvent(d.side, d.fork, 0)) != cudaSuccess) return cuda_status(e);
            credit_args fa = *a;
            const long long ld_in = a->ld_in ? a->ld_in : a->cols, ld_out = a->ld_out ? a->ld_out : a->cols;
            fa.in = static_cast<const unsigned char *>(a->in) + n_cl * ld_in * isz;
            fa.out = lse ? static_cast<void *>(static_cast<unsigned char *>(a->out) + n_cl * 4)
                         : static_cast<void *>(static_cast<unsigned char *>(a->out) + n_cl * ld_out * osz);
            if (a->in_scale) fa.in_scale = a->in_scale + n_cl;
            if (a->out_scale) fa.out_scale = a->out_scale + n_cl;
            fa.rows = n_fill;
            credit_plan_t fp{};
            fp.path = CREDIT_PATH_TWO_PASS;
            fp.cluster_size = 1;
            fp.ctas_per_row = p->fill_g > 0 ? p->fill_g : fill_split(a->cols, isz);
            const credit_status st2 = run_with_plan(device, &fa, &fp, d.side);
            if (st2 != CREDIT_OK) return st2;
            if ((e = cudaEventRecord(d.join, d.side)) != cudaSuccess) return cuda_status(e);
            if ((e = cudaStreamWaitEvent(s, d.join, 0)) != cudaSuccess) return cuda_status(e);
        }
        return CREDIT_OK;
    }

    // TWO_PASS.  Default CTA: 512 threads for FP32 rows, 256 for BF16 / FP8 rows (more CTAs per SM keep
    // more loads in flight: softmax / log-sum-exp over 4096 x 128K-256K BF16 and FP8 rows measured 6-13%
    // faster than with 512, 1024 slower still)
    const int G = p->ctas_per_row;
    const int threads = p->threads ? p->threads : (isz <= 2 ? 256 : 512);
    if (G == 1) {
        credit_status st = prepare_kernel(d, ks.tp_fused, false);
        if (st != CREDIT_OK) return st;
        const long long max_rows = 0x7FFFFFFFLL;
        for (long long r0 = 0; r0 < rows; r0 += max_rows) {
            const long long n = rows - r0 < max_rows ? rows - r0 : max_rows;
            RowArgs r = rows_from(base, r0, n, isz, osz, lse);
            void *args[] = {&r};
            cudaError_t e = launch(ks.tp_fused, dim3(static_cast<unsigned>(n)), dim3(threads), 0, 1, s, args);
            if (e != cudaSuccess) return cuda_status(e);
            g_launch_count.fetch_add(1);
        }
        return CREDIT_OK;
    }
    const long long cap_rows = static_cast<long long>(d.info.ws_floats / (static_cast<size_t>(G) * 4));
    const long long max_rows = cap_rows < 0x7FFFFFFFLL / G ? cap_rows : 0x7FFFFFFFLL / G;
    const bool fp8_stage = (a->op == OP_LN || a->op == OP_RMS) && tout == DT_E4M3;
    for (long long r0 = 0; r0 < rows; r0 += max_rows) {
        const long long n = rows - r0 < max_rows ? rows - r0 : max_rows;
        RowArgs r = rows_from(base, r0, n, isz, osz, lse);
        r.G = G;
        void *args[] = {&r};
        const dim3 grid(static_cast<unsigned>(G * n));
        cudaError_t e = launch(ks.tp_stats, grid, dim3(threads), 0, 1, s, args);
        if (e != cudaSuccess) return cuda_status(e);
        g_launch_count.fetch_add(1);
        if (lse) {
            long long nn = n;
            void *args2[] = {&r, &nn};
            e = launch(ks.tp_lse_final, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, 1, s, args2);
            if (e != cudaSuccess) return cuda_status(e);
            g_launch_count.fetch_add(1);
            continue;
        }
        if (fp8_stage) {
            e = launch(ks.tp_amax, grid, dim3(threads), 0, 1, s, args);
            if (e != cudaSuccess) return cuda_status(e);
            g_launch_count.fetch_add(1);
        }
        e = launch(ks.tp_apply, grid, dim3(threads), 0, 1, s, args);
        if (e != cudaSuccess) return cuda_status(e);
        g_launch_count.fetch_add(1);
    }
    return CREDIT_OK;
}

credit_status ensure_init(int *device_out, cudaStream_t s) {
    const int dev = current_device();
    if (dev < 0 || dev >= kMaxDevices) return CREDIT_ERR_CUDA;
    *device_out = dev;
    if (g_dev[dev].ready.load()) return CREDIT_OK;
    if (stream_capturing(s)) return CREDIT_ERR_CAPTURE;  // init allocates
    return credit_init(dev);
}

}  // namespace credit

extern "C" {

credit_status credit_run_ex(const credit_args *args, const credit_plan_t *plan, cudaStream_t stream) {
    credit_status st = validate_args(args);
    if (st != CREDIT_OK) return st;
    if (args->rows == 0) return CREDIT_OK;
    int dev = 0;
    if ((st = ensure_init(&dev, stream)) != CREDIT_OK) return st;
    credit_plan_t chosen;
    if (plan) {
        chosen = *plan;
    } else {
        st = credit_plan_ex(static_cast<credit_op>(args->op), args->rows, args->cols,
                            static_cast<credit_dtype>(args->in_dtype),
                            static_cast<credit_dtype>(args->op == OP_LSE ? DT_F32 : args->out_dtype), &chosen);
        if (st != CREDIT_OK) return st;
    }
    if ((st = check_plan(dev, args, &chosen)) != CREDIT_OK) return st;
    return run_with_plan(dev, args, &chosen, stream);
}

credit_status credit_set_trace(void *device_buf, int64_t bytes) {
    if (device_buf == nullptr || bytes <= 0) {
        g_trace_buf = nullptr;
        g_trace_rows = 0;
        return CREDIT_OK;
    }
    const int64_t per_row = static_cast<int64_t>(kTraceCtas) * kTraceFields * 8;
    if (reinterpret_cast<uintptr_t>(device_buf) % 8 || bytes < per_row) return CREDIT_ERR_INVALID_ARG;
    g_trace_buf = static_cast<unsigned long long *>(device_buf);
    g_trace_rows = static_cast<int>(bytes / per_row);
    return CREDIT_OK;
}

credit_status credit_set_wait_test(int64_t wait_ns, int32_t extra_tx_bytes) {
    if (wait_ns < 0 || extra_tx_bytes < 0 || extra_tx_bytes % 16 || extra_tx_bytes > (1 << 20))
        return CREDIT_ERR_INVALID_ARG;
    g_wait_ns.store(static_cast<unsigned long long>(wait_ns));
    g_test_extra_tx.store(extra_tx_bytes);
    return CREDIT_OK;
}

int32_t credit_max_clusters(const credit_args *args, const credit_plan_t *plan) {
    if (!plan || validate_args(args) != CREDIT_OK) return 0;
    if (plan->path != CREDIT_PATH_ONE_CTA && plan->path != CREDIT_PATH_CLUSTER) return 0;
    int dev = 0;
    if (ensure_init(&dev, nullptr) != CREDIT_OK) return 0;
    if (check_plan(dev, args, plan) != CREDIT_OK) return 0;
    const DeviceInfo *di = device_info(dev);
    const int P = plan->path == CREDIT_PATH_ONE_CTA ? 1 : plan->cluster_size;
    RingCfg rc;
    if (!ring_config_for(*di, args, dtype_size(args->in_dtype), P, plan, &rc)) return 0;
    const int tout = args->op == OP_LSE ? DT_F32 : args->out_dtype;
    return ring_max_clusters(dev, args->op, args->in_dtype, tout, P, rc.threads, rc.smem, rc.tmem != 0);
}

credit_status credit_plan_check(const credit_args *args, const credit_plan_t *plan) {
    credit_status st = validate_args(args);
    if (st != CREDIT_OK) return st;
    if (!plan) return CREDIT_ERR_INVALID_ARG;
    int dev = 0;
    if ((st = ensure_init(&dev, nullptr)) != CREDIT_OK) return st;
    return check_plan(dev, args, plan);
}

static credit_status simple(credit_op op, const void *in, void *out, int64_t rows, int64_t cols, credit_dtype dtype,
                            cudaStream_t stream) {
    if (dtype == CREDIT_FP8_E4M3) return CREDIT_ERR_INVALID_ARG;  // scales need credit_run_ex
    credit_args a;
    std::memset(&a, 0, sizeof(a));
    a.op = op;
    a.in = in;
    a.out = out;
    a.rows = rows;
    a.cols = cols;
    a.in_dtype = dtype;
    a.out_dtype = op == CREDIT_OP_LOGSUMEXP ? CREDIT_F32 : dtype;
    a.eps = -1.0f;
    return credit_run_ex(&a, nullptr, stream);
}

credit_status credit_softmax(const void *in, void *out, int64_t rows, int64_t cols, credit_dtype dtype,
                             cudaStream_t stream) {
    return simple(CREDIT_OP_SOFTMAX, in, out, rows, cols, dtype, stream);
}
credit_status credit_logsumexp(const void *in, void *out, int64_t rows, int64_t cols, credit_dtype dtype,
                               cudaStream_t stream) {
    return simple(CREDIT_OP_LOGSUMEXP, in, out, rows, cols, dtype, stream);
}
credit_status credit_layernorm(const void *in, void *out, int64_t rows, int64_t cols, credit_dtype dtype,
                               cudaStream_t stream) {
    return simple(CREDIT_OP_LAYERNORM, in, out, rows, cols, dtype, stream);
}
credit_status credit_rmsnorm(const void *in, void *out, int64_t rows, int64_t cols, credit_dtype dtype,
                             cudaStream_t stream) {
    return simple(CREDIT_OP_RMSNORM, in, out, rows, cols, dtype, stream);
}

// Number of kernel launches this library has issued in this process (all
// devices).  Lets a caller count the launches inside a timed region.
long long credit_launch_count(void) { return g_launch_count.load(); }

}  // extern "C"
