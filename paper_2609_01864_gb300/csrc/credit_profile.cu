// credit_profile.cu -- primitive characterisation and the control kernel
// (CREDIT Sec. III-A, Table II; Sec. III-D, T_ctrl).
//
// K1  latency: a dependent chain of shared-memory loads, local and remote
//     (DSMEM, ld.shared::cluster), cycles per load.
// K2  throughput: many independent 16-byte loads / stores, local and remote,
//     bytes per cycle per SM; the remote-store rate is measured for every
//     cluster size P (B_DSM^w(P) of Eq. 8).
// K3  cluster synchronisation: cycles per barrier.cluster arrive + wait.
// K4  control: the ring kernel's launch (same grid, cluster size, threads and
//     dynamic shared memory) and per-row synchronisation (one DSMEM push
//     all-gather per stage) with no data work.  T_ctrl(M, N, P) is its time
//     minus the time of the same kernel at P = 1 (Sec. III-D).
// The two CTAs of a latency / throughput cluster each take more than half of
// an SM's shared memory, so they run on different SMs (checked with %smid).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/credit.h"
#include "credit_host.h"
#include "credit_rows.cuh"

using namespace credit;

namespace {

__device__ __forceinline__ uint32_t smid() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t ld_shared_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// out[0] = cycles per dependent load (local), out[1] = (remote), out[2..3] = smid of CTA 0/1
__global__ void k_latency(unsigned long long *out, int n_nodes, int iters) {
    extern __shared__ __align__(16) uint32_t chain[];
    const uint32_t rank = cluster_ctarank();
    // a random cycle: node i -> (i * 97 + 13) mod n_nodes (n_nodes prime to 97)
    for (int i = threadIdx.x; i < n_nodes; i += blockDim.x)
        chain[i] = smem_addr(&chain[(static_cast<long long>(i) * 97 + 13) % n_nodes]);
    cluster_arrive_release();
    cluster_wait_acquire();
    if (rank == 0 && threadIdx.x == 0) {
        uint32_t p = smem_addr(&chain[0]);
        for (int i = 0; i < 64; ++i) p = ld_shared_u32(p);  // warm
        long long t0 = clock64();
        for (int i = 0; i < iters; ++i) p = ld_shared_u32(p);
        long long t1 = clock64();
        // remote: follow the same chain inside CTA 1's shared memory
        uint32_t q = mapa_shared(smem_addr(&chain[0]), 1);
        const uint32_t base_local = smem_addr(&chain[0]), base_remote = q;
        for (int i = 0; i < 64; ++i) q = mapa_shared(ld_cluster_u32(q), 1);
        long long t2 = clock64();
        for (int i = 0; i < iters; ++i) q = mapa_shared(ld_cluster_u32(q), 1);
        long long t3 = clock64();
        (void)base_local;
        (void)base_remote;
        out[0] = static_cast<unsigned long long>(t1 - t0);
        out[1] = static_cast<unsigned long long>(t3 - t2);
        out[4] = p + q;  // keep the chains live
    }
    if (threadIdx.x == 0) out[2 + rank] = smid();
    cluster_arrive_release();
    cluster_wait_acquire();
}

// mode 0 local read, 1 local store, 2 remote read (peer rank+1), 3 remote store
// (round-robin over the P-1 peers).  out[blockIdx] = cycles, bytes in out2.
__global__ void k_throughput(unsigned long long *cycles, int mode, int iters, int buf_bytes) {
    extern __shared__ __align__(16) unsigned char buf[];
    const uint32_t rank = cluster_ctarank(), P = cluster_nctarank();
    const int n16 = buf_bytes / 16;
    for (int i = threadIdx.x; i < n16; i += blockDim.x)
        reinterpret_cast<uint4 *>(buf)[i] = make_uint4(i, i + 1, i + 2, i + 3);
    cluster_arrive_release();
    cluster_wait_acquire();
    __syncthreads();
    const uint32_t base = smem_addr(buf);
    uint32_t acc = 0;
    long long t0 = clock64();
    if (mode == 0) {
        for (int it = 0; it < iters; ++it)
            for (int i = threadIdx.x; i < n16; i += blockDim.x) {
                uint4 v;
                asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "r"(base + 16 * i)
                             : "memory");
                acc += v.x ^ v.w;
            }
    } else if (mode == 1) {
        for (int it = 0; it < iters; ++it)
            for (int i = threadIdx.x; i < n16; i += blockDim.x)
                asm volatile("st.shared.v4.u32 [%0], {%1,%1,%1,%1};" ::"r"(base + 16 * i), "r"(it) : "memory");
    } else if (mode == 2) {
        const uint32_t rb = mapa_shared(base, (rank + 1) % P);
        for (int it = 0; it < iters; ++it)
            for (int i = threadIdx.x; i < n16; i += blockDim.x) {
                uint4 v;
                asm volatile("ld.shared::cluster.v4.u32 {%0,%1,%2,%3}, [%4];"
                             : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                             : "r"(rb + 16 * i)
                             : "memory");
                acc += v.x ^ v.w;
            }
    } else {
        for (int it = 0; it < iters; ++it) {
            const uint32_t peer = (rank + 1 + static_cast<uint32_t>(it) % (P - 1)) % P;
            const uint32_t rb = mapa_shared(base, peer);
            for (int i = threadIdx.x; i < n16; i += blockDim.x)
                asm volatile("st.shared::cluster.v4.u32 [%0], {%1,%1,%1,%1};" ::"r"(rb + 16 * i), "r"(it) : "memory");
        }
    }
    __syncthreads();
    long long t1 = clock64();
    cluster_arrive_release();
    cluster_wait_acquire();
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(t1 - t0);
    if (acc == 0x12345678u) cycles[gridDim.x] = acc;  // keep loads live
}

__global__ void k_sync(unsigned long long *cycles, int iters) {
    cluster_arrive_release();
    cluster_wait_acquire();
    long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        cluster_arrive_release();
        cluster_wait_acquire();
    }
    long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<unsigned long long>(t1 - t0);
}

// SM clock under load: cycles counted by one thread while the host times the
// kernel with events.
__global__ void k_clock(unsigned long long *cycles, long long spin) {
    long long t0 = clock64();
    while (clock64() - t0 < spin) {
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) cycles[0] = static_cast<unsigned long long>(clock64() - t0);
}

// K4: the ring kernel's synchronisation skeleton without data.  Launch shape
// as k_ring (persistent clusters, producer + reducers + writers, same dynamic
// shared memory); per row the reducers run the DSMEM push all-gather (stages
// times) and hand the row to the writers through the stats mbarriers.
__global__ void __launch_bounds__(288, 3) k_control(const RowArgs a, int stages) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *xbar = full + 64;
    uint64_t *stats_full = full + 68;
    uint64_t *stats_empty = full + 70;
    float *slots = reinterpret_cast<float *>(smem + 1152);
    const int P = static_cast<int>(cluster_nctarank());
    const int c = P > 1 ? static_cast<int>(cluster_ctarank()) : 0;
    const long long ncl = gridDim.x / P, cl = blockIdx.x / P;
    const int tid = threadIdx.x, Tr = a.reducers, Tp = static_cast<int>(blockDim.x) - 32, Tw = Tp - Tr;
    const int Ww = Tw >> 5;
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) mbar_init(&xbar[k], 1);
        for (int k = 0; k < 2; ++k) {
            mbar_init(&stats_full[k], 1);
            mbar_init(&stats_empty[k], static_cast<uint32_t>(Ww));
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (P > 1) cluster_arrive_release();
    bool waited = false;
    if (tid < Tr) {
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const int par = rr & 1;
            const uint32_t xphase = static_cast<uint32_t>((rr >> 1) & 1);
            float v = static_cast<float>(row);
            if (P > 1) {
                if (!waited) {
                    cluster_wait_acquire();
                    waited = true;
                }
                for (int st = 0; st < stages; ++st) {
                    const float *sl = exchange_push<2>(v, v, slots, xbar, st, par, xphase, P, c, Tr, a.err);
                    v += sl[0];
                }
            }
            if (tid == 0) {
                if (rr >= 2) mbar_wait_bounded(&stats_empty[par], static_cast<uint32_t>(((rr >> 1) - 1) & 1), a.err);
                mbar_arrive(&stats_full[par]);
            }
        }
    } else if (tid < Tp) {
        const int wt = tid - Tr;
        int rr = 0;
        for (long long row = cl; row < a.rows; row += ncl, ++rr) {
            const int par = rr & 1;
            mbar_wait_bounded(&stats_full[par], static_cast<uint32_t>((rr >> 1) & 1), a.err);
            __syncwarp();
            if ((wt & 31) == 0) mbar_arrive(&stats_empty[par]);
        }
    }
    (void)full;
    if (P > 1) {
        if (!waited) cluster_wait_acquire();
        cluster_arrive_release();
        cluster_wait_acquire();
    }
}

cudaError_t launch_cluster(const void *fn, unsigned grid, unsigned block, size_t smem, int P, cudaStream_t s,
                           void **args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = P;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, fn, args);
}

template <class T>
T median(std::vector<T> v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? T() : v[v.size() / 2];
}

}  // namespace

extern "C" {

credit_status credit_microbench(credit_microbench_t *out, int runs) {
    if (!out) return CREDIT_ERR_INVALID_ARG;
    if (runs < 1) runs = 15;
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    const DeviceInfo *di = device_info(dev);
    std::memset(out, 0, sizeof(*out));
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, 64 * sizeof(unsigned long long)) != cudaSuccess) return CREDIT_ERR_CUDA;
    const int big = static_cast<int>(di->smem_optin);  // > half an SM: two CTAs never share one
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(k_latency, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_throughput, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_throughput, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sync, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
        cudaFree(d);
        return CREDIT_ERR_CUDA;
    }
    std::vector<double> lat_l, lat_r;
    unsigned long long h[8];
    const int iters = 4096, nodes = 4093;  // 4093 is prime
    for (int r = 0; r < runs && e == cudaSuccess; ++r) {
        int it = iters, nn = nodes;
        void *args[] = {&d, &nn, &it};
        e = launch_cluster(reinterpret_cast<const void *>(k_latency), 2, 32, big, 2, nullptr, args);
        if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) break;
        lat_l.push_back(static_cast<double>(h[0]) / iters);
        lat_r.push_back(static_cast<double>(h[1]) / iters);
        out->distinct_sms = h[2] != h[3] ? 1 : 0;
    }
    out->lat_local_cycles = median(lat_l);
    out->lat_remote_cycles = median(lat_r);
    // throughput: one cluster of 2 for reads / local store; every P for remote store
    const int tb_bytes = 128 * 1024, tb_iters = 16, tb_threads = 512;
    auto rate = [&](int mode, int P, double *res) -> cudaError_t {
        std::vector<double> v;
        for (int r = 0; r < runs; ++r) {
            int m = mode, it = tb_iters, bb = tb_bytes;
            void *args[] = {&d, &m, &it, &bb};
            cudaError_t ee =
                launch_cluster(reinterpret_cast<const void *>(k_throughput), P, tb_threads, big, P, nullptr, args);
            if (ee == cudaSuccess) ee = cudaMemcpy(h, d, sizeof(unsigned long long) * (P < 8 ? P : 8),
                                                   cudaMemcpyDeviceToHost);
            if (ee != cudaSuccess) return ee;
            const double cyc = static_cast<double>(h[0]);
            v.push_back(static_cast<double>(tb_bytes) * tb_iters / cyc);
        }
        *res = median(v);
        return cudaSuccess;
    };
    if (e == cudaSuccess) e = rate(0, 2, &out->rate_local_read);
    if (e == cudaSuccess) e = rate(1, 2, &out->rate_local_store);
    if (e == cudaSuccess) e = rate(2, 2, &out->rate_remote_read);
    const int Ps[4] = {2, 4, 8, 16};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = rate(3, Ps[k], &out->rate_remote_store[k]);
    // cluster sync cycles per P
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        std::vector<double> v;
        for (int r = 0; r < runs && e == cudaSuccess; ++r) {
            int it = 1000;
            void *args[] = {&d, &it};
            e = launch_cluster(reinterpret_cast<const void *>(k_sync), Ps[k], 128, 0, Ps[k], nullptr, args);
            if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
            v.push_back(static_cast<double>(h[0]) / 1000.0);
        }
        out->sync_cycles[k] = median(v);
    }
    // SM clock under load (all SMs spinning), MHz
    if (e == cudaSuccess) {
        cudaEvent_t a0, a1;
        cudaEventCreate(&a0);
        cudaEventCreate(&a1);
        long long spin = 200000000LL;  // ~0.1 s at 2 GHz
        void *args[] = {&d, &spin};
        cudaEventRecord(a0);
        e = cudaLaunchKernel(reinterpret_cast<const void *>(k_clock), dim3(di->sm_count * 4), dim3(128), args, 0,
                             nullptr);
        cudaEventRecord(a1);
        if (e == cudaSuccess) e = cudaEventSynchronize(a1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a0, a1);
        if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
        out->sm_clock_mhz = ms > 0.0f ? static_cast<double>(h[0]) / (ms * 1e3) : 0.0;
        cudaEventDestroy(a0);
        cudaEventDestroy(a1);
    }
    cudaFree(d);
    return e == cudaSuccess ? CREDIT_OK : CREDIT_ERR_CUDA;
}

credit_status credit_control_time(credit_op op, int64_t rows, int64_t cols, credit_dtype dtype, int32_t P,
                                  int32_t reps, float *us_out) {
    if (!us_out || rows <= 0 || cols <= 0 || P < 1 || P > 16 || dtype < 0 || dtype > 2) return CREDIT_ERR_INVALID_ARG;
    if (reps < 1) reps = 15;
    int dev = 0;
    credit_status st = ensure_init(&dev, nullptr);
    if (st != CREDIT_OK) return st;
    const DeviceInfo *di = device_info(dev);
    RingCfg rc;
    if (!ring_config(*di, cols, dtype_size(dtype), P, 0, 0, 0, 0, 0, &rc)) return CREDIT_ERR_UNSUPPORTED;
    const int tout = op == CREDIT_OP_LOGSUMEXP ? 0 : dtype;
    const int maxc = ring_max_clusters(dev, op, dtype, tout, P, rc.threads, rc.smem);
    if (maxc <= 0) return CREDIT_ERR_UNSUPPORTED;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_control, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(di->smem_optin)) != cudaSuccess ||
            cudaFuncSetAttribute(k_control, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            return CREDIT_ERR_CUDA;
        attr_set = true;
    }
    unsigned *err = nullptr;
    if (cudaMalloc(&err, 16) != cudaSuccess) return CREDIT_ERR_CUDA;
    cudaMemset(err, 0, 16);
    RowArgs r{};
    r.rows = rows;
    r.cols = cols;
    r.reducers = rc.reducers;
    r.err = err;
    int stages = (op == CREDIT_OP_LAYERNORM || op == CREDIT_OP_RMSNORM) && dtype == CREDIT_FP8_E4M3 ? 2 : 1;
    const long long ncl = rows < maxc ? rows : maxc;
    void *args[] = {&r, &stages};
    cudaEvent_t a0, a1;
    cudaEventCreate(&a0);
    cudaEventCreate(&a1);
    std::vector<float> v;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < reps + 2 && e == cudaSuccess; ++k) {
        cudaEventRecord(a0);
        if (P > 1) {
            e = launch_cluster(reinterpret_cast<const void *>(k_control), static_cast<unsigned>(P * ncl), rc.threads,
                               rc.smem, P, nullptr, args);
        } else {
            e = cudaLaunchKernel(reinterpret_cast<const void *>(k_control), dim3(static_cast<unsigned>(ncl)),
                                 dim3(rc.threads), args, static_cast<size_t>(rc.smem), nullptr);
        }
        cudaEventRecord(a1);
        if (e == cudaSuccess) e = cudaEventSynchronize(a1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a0, a1);
        if (k >= 2) v.push_back(ms * 1e3f);
    }
    unsigned herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
    cudaFree(err);
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    if (e != cudaSuccess) return CREDIT_ERR_CUDA;
    if (herr) return CREDIT_ERR_TIMEOUT;
    *us_out = median(v);
    return CREDIT_OK;
}

}  // extern "C"
