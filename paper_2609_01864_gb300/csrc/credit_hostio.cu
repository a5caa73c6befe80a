// credit_hostio.cu -- credit_run_host: one op on host buffers, with the rows
// streamed through device staging buffers.
//
// The rows are cut into blocks; block b's input is copied in on the h2d
// stream, the op runs on the compute stream, and the output is copied out on
// the d2h stream (by a copy kernel of the library when the host buffer is
// pinned, else by the copy engines).  kBlocks staging slots rotate, so the copy-in of block
// b + 1, the op on block b and the copy-out of block b - 1 run at the same
// time (the host link is full duplex; the op itself takes a few percent of
// the copy time).  Events order the three streams:
//   copy-in b     waits for copy-out b - kBlocks (its slot is free again)
//   op b          waits for copy-in b
//   copy-out b    waits for op b
// The staging slots are allocated on first use and kept per device (grown
// when a larger block is needed), like the two-pass workspace.
#include <cuda_runtime.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "../../include/credit.h"
#include "credit_host.h"

namespace credit {
extern std::atomic<long long> g_launch_count;
namespace {

constexpr int kBlocks = 3;                            // staging slots in rotation
constexpr long long kBlockBytes = 256LL << 20;        // largest block (input or output bytes)
constexpr int kMinBlocksPerCall = 8;                  // aim for this many blocks, for overlap
constexpr int kMaxDevices = 64;

struct HostIO {
    std::mutex mu;
    bool ready = false;
    cudaStream_t s_in = nullptr, s_op = nullptr, s_out = nullptr;
    cudaEvent_t in_done[kBlocks], op_done[kBlocks], out_done[kBlocks];
    unsigned char *in_buf[kBlocks] = {}, *out_buf[kBlocks] = {};
    float *isc[kBlocks] = {}, *osc[kBlocks] = {};
    float *affine = nullptr;  // gamma, then beta at the next 256-byte boundary
    size_t in_cap = 0, out_cap = 0, rows_cap = 0, cols_cap = 0;
};
HostIO g_io[kMaxDevices];

cudaError_t io_init(HostIO &io) {
    if (io.ready) return cudaSuccess;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&io.s_in, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&io.s_op, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&io.s_out, cudaStreamNonBlocking)) != cudaSuccess) return e;
    for (int k = 0; k < kBlocks; ++k) {
        if ((e = cudaEventCreateWithFlags(&io.in_done[k], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&io.op_done[k], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&io.out_done[k], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    io.ready = true;
    return cudaSuccess;
}

// Grow-only device buffers (the streams are idle when this runs).
template <class T>
cudaError_t grow(T **p, size_t bytes) {
    if (*p) cudaFree(*p);
    *p = nullptr;
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}

cudaError_t io_reserve(HostIO &io, size_t in_bytes, size_t out_bytes, size_t rows, size_t cols) {
    cudaError_t e;
    if (in_bytes > io.in_cap || out_bytes > io.out_cap || rows > io.rows_cap) {
        for (int k = 0; k < kBlocks; ++k) {
            if (in_bytes > io.in_cap && (e = grow(&io.in_buf[k], in_bytes)) != cudaSuccess) return e;
            if (out_bytes > io.out_cap && (e = grow(&io.out_buf[k], out_bytes)) != cudaSuccess) return e;
            if (rows > io.rows_cap) {
                if ((e = grow(&io.isc[k], rows * 4)) != cudaSuccess) return e;
                if ((e = grow(&io.osc[k], rows * 4)) != cudaSuccess) return e;
            }
        }
        if (in_bytes > io.in_cap) io.in_cap = in_bytes;
        if (out_bytes > io.out_cap) io.out_cap = out_bytes;
        if (rows > io.rows_cap) io.rows_cap = rows;
    }
    if (cols > io.cols_cap) {
        if ((e = grow(&io.affine, (cols + 64) * 8)) != cudaSuccess) return e;
        io.cols_cap = cols;
    }
    return cudaSuccess;
}

credit_status status_of(cudaError_t e) { return e == cudaSuccess ? CREDIT_OK : CREDIT_ERR_CUDA; }

// ---------------------------------------------------------------- SM-driven copies
// Blocks of pinned host rows move between host memory and the staging slots
// in a copy kernel: the SMs load and store through the host link themselves
// instead of handing the transfer to the copy engines.  On GB300 both reach
// the link's rate in one direction (211 GB/s in, 193 out), but with both
// directions busy at once the copy engines fell to 117 GB/s on a box that had
// just run a long GPU job, where copy kernels kept 250-295 GB/s.
constexpr int kCopyCtas = 76;     // per copy: two of them (in and out) fill half the SMs' thread slots
constexpr int kCopyThreads = 256;

// One contiguous range of n words W.  Built for at most 40 registers, so a
// copy CTA fits on an SM beside a k_ring_tm CTA (576 threads x 96 registers):
// the op of one block runs while the copies of its neighbours do.
template <typename W>
__global__ void __launch_bounds__(kCopyThreads, 6) k_copy_1d(const W *__restrict__ src, W *__restrict__ dst,
                                                            long long n) {
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {  // two independent loads in flight per thread
        const W a = src[i], b = src[i + stride];
        dst[i] = a;
        dst[i + stride] = b;
    }
    for (; i < n; i += stride) dst[i] = src[i];
}

// rows rows of `words` words W each, at their own pitches (bytes); a CTA per row at a time.
template <typename W>
__global__ void __launch_bounds__(kCopyThreads, 6) k_copy_2d(const unsigned char *__restrict__ src, long long src_pitch,
                                                        unsigned char *__restrict__ dst, long long dst_pitch,
                                                        long long rows, long long words) {
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const W *s = reinterpret_cast<const W *>(src + r * src_pitch);
        W *d = reinterpret_cast<W *>(dst + r * dst_pitch);
        for (long long k = threadIdx.x; k < words; k += blockDim.x) d[k] = s[k];
    }
}

// rows x row_bytes from src (pitch sp) to dst (pitch dp) on `stream`, both
// addresses device-accessible: 16-byte words where every address, pitch and
// the row length allow it, else 4-byte words, else bytes.
cudaError_t launch_copy(const void *src, long long sp, void *dst, long long dp, long long rows, long long row_bytes,
                        cudaStream_t stream) {
    if (rows <= 0 || row_bytes <= 0) return cudaSuccess;
    const bool dense = rows == 1 || (sp == row_bytes && dp == row_bytes);
    const uintptr_t bits = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                           static_cast<uintptr_t>(row_bytes) | (dense ? 0 : static_cast<uintptr_t>(sp | dp));
    const int w = (bits & 15u) == 0 ? 16 : ((bits & 3u) == 0 ? 4 : 1);
    if (dense) {
        const long long n = rows * row_bytes / w;
        if (w == 16)
            k_copy_1d<uint4><<<kCopyCtas, kCopyThreads, 0, stream>>>(static_cast<const uint4 *>(src),
                                                                     static_cast<uint4 *>(dst), n);
        else if (w == 4)
            k_copy_1d<uint32_t><<<kCopyCtas, kCopyThreads, 0, stream>>>(static_cast<const uint32_t *>(src),
                                                                        static_cast<uint32_t *>(dst), n);
        else
            k_copy_1d<unsigned char><<<kCopyCtas, kCopyThreads, 0, stream>>>(static_cast<const unsigned char *>(src),
                                                                             static_cast<unsigned char *>(dst), n);
    } else {
        const auto *s8 = static_cast<const unsigned char *>(src);
        auto *d8 = static_cast<unsigned char *>(dst);
        if (w == 16) k_copy_2d<uint4><<<kCopyCtas, kCopyThreads, 0, stream>>>(s8, sp, d8, dp, rows, row_bytes / 16);
        else if (w == 4) k_copy_2d<uint32_t><<<kCopyCtas, kCopyThreads, 0, stream>>>(s8, sp, d8, dp, rows, row_bytes / 4);
        else k_copy_2d<unsigned char><<<kCopyCtas, kCopyThreads, 0, stream>>>(s8, sp, d8, dp, rows, row_bytes);
    }
    g_launch_count.fetch_add(1);
    return cudaGetLastError();
}

// The device address of host range [p, p + bytes) if the GPU may load / store
// it directly (page-locked or registered memory, first and last byte), else
// nullptr: such ranges are copied by the copy engines (cudaMemcpy*Async).
const unsigned char *device_view(const void *p, long long bytes) {
    if (p == nullptr || bytes <= 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
        cudaPointerGetAttributes(&b, static_cast<const unsigned char *>(p) + bytes - 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || a.devicePointer == nullptr ||
        b.devicePointer == nullptr)
        return nullptr;
    return static_cast<const unsigned char *>(a.devicePointer);
}

}  // namespace
}  // namespace credit

using namespace credit;

extern "C" credit_status credit_run_host(const credit_args *args, const credit_plan_t *plan) {
    credit_status st = validate_args(args);
    if (st != CREDIT_OK) return st;
    if (args->rows == 0) return CREDIT_OK;
    int dev = 0;
    if ((st = ensure_init(&dev, nullptr)) != CREDIT_OK) return st;
    if (dev >= kMaxDevices) return CREDIT_ERR_UNSUPPORTED;
    HostIO &io = g_io[dev];
    std::lock_guard<std::mutex> lk(io.mu);  // one host call per device at a time
    if ((st = status_of(io_init(io))) != CREDIT_OK) return st;

    const bool lse = args->op == CREDIT_OP_LOGSUMEXP;
    const int tin = args->in_dtype, tout = lse ? CREDIT_F32 : args->out_dtype;
    const long long isz = dtype_size(tin), osz = dtype_size(tout);
    const long long rows = args->rows, cols = args->cols;
    const long long ld_in = args->ld_in ? args->ld_in : cols, ld_out = args->ld_out ? args->ld_out : cols;
    const long long row_in = cols * isz, row_out = lse ? 4 : cols * osz;
    const long long row_max = row_in > row_out ? row_in : row_out;
    // block rows: about rows / kMinBlocksPerCall, at most kBlockBytes per buffer
    long long br = (rows + kMinBlocksPerCall - 1) / kMinBlocksPerCall;
    if (br * row_max > kBlockBytes) br = kBlockBytes / row_max;
    if (br < 1) br = 1;
    if ((st = status_of(io_reserve(io, static_cast<size_t>(br * row_in), static_cast<size_t>(br * row_out),
                                   static_cast<size_t>(br), static_cast<size_t>(cols)))) != CREDIT_OK)
        return st;

    // gamma / beta once per call (host -> device, on the op stream)
    const bool norm = args->op == CREDIT_OP_LAYERNORM || args->op == CREDIT_OP_RMSNORM;
    const float *d_gamma = nullptr, *d_beta = nullptr;
    if (norm && args->gamma) {
        if ((st = status_of(cudaMemcpyAsync(io.affine, args->gamma, cols * 4, cudaMemcpyHostToDevice, io.s_op))) !=
            CREDIT_OK)
            return st;
        d_gamma = io.affine;
    }
    if (args->op == CREDIT_OP_LAYERNORM && args->beta) {
        float *bd = io.affine + (cols + 63) / 64 * 64;
        if ((st = status_of(cudaMemcpyAsync(bd, args->beta, cols * 4, cudaMemcpyHostToDevice, io.s_op))) !=
            CREDIT_OK)
            return st;
        d_beta = bd;
    }

    // one plan for the block shape (the caller's, or the planner's), checked
    // before anything moves
    credit_args blk = *args;
    blk.in = io.in_buf[0];
    blk.out = io.out_buf[0];
    blk.rows = br;
    blk.ld_in = 0;
    blk.ld_out = 0;
    blk.in_scale = tin == CREDIT_FP8_E4M3 ? io.isc[0] : nullptr;
    blk.out_scale = (!lse && (tout == CREDIT_FP8_E4M3 || tout == CREDIT_INT8)) ? io.osc[0] : nullptr;
    blk.gamma = d_gamma;
    blk.beta = d_beta;
    credit_plan_t chosen;
    if (plan) {
        chosen = *plan;
    } else if ((st = credit_plan_ex(static_cast<credit_op>(args->op), br, cols, static_cast<credit_dtype>(tin),
                                    static_cast<credit_dtype>(tout), &chosen)) != CREDIT_OK) {
        return st;
    }
    if ((st = check_plan(dev, &blk, &chosen)) != CREDIT_OK) return st;

    const unsigned char *hin = static_cast<const unsigned char *>(args->in);
    unsigned char *hout = static_cast<unsigned char *>(args->out);
    // pinned row buffers move by copy kernels (launch_copy), pageable ones by the copy engines
    const long long in_span = (rows - 1) * ld_in * isz + row_in;
    const long long out_span = lse ? rows * 4 : (rows - 1) * ld_out * osz + row_out;
    const unsigned char *din = device_view(hin, in_span);
    unsigned char *dout = const_cast<unsigned char *>(device_view(hout, out_span));
    cudaError_t e = cudaSuccess;
    long long b = 0;
    for (long long r0 = 0; r0 < rows && e == cudaSuccess; r0 += br, ++b) {
        const int k = static_cast<int>(b % kBlocks);
        const long long n = rows - r0 < br ? rows - r0 : br;
        // copy-in (slot k free once its previous copy-out finished)
        if (b >= kBlocks && (e = cudaStreamWaitEvent(io.s_in, io.out_done[k], 0)) != cudaSuccess) break;
        if (din)
            e = launch_copy(din + r0 * ld_in * isz, ld_in * isz, io.in_buf[k], row_in, n, row_in, io.s_in);
        else if (ld_in * isz == row_in)  // contiguous rows: one plain copy
            e = cudaMemcpyAsync(io.in_buf[k], hin + r0 * row_in, n * row_in, cudaMemcpyHostToDevice, io.s_in);
        else
            e = cudaMemcpy2DAsync(io.in_buf[k], row_in, hin + r0 * ld_in * isz, ld_in * isz, row_in, n,
                                  cudaMemcpyHostToDevice, io.s_in);
        if (e == cudaSuccess && tin == CREDIT_FP8_E4M3)
            e = cudaMemcpyAsync(io.isc[k], args->in_scale + r0, n * 4, cudaMemcpyHostToDevice, io.s_in);
        if (e == cudaSuccess) e = cudaEventRecord(io.in_done[k], io.s_in);
        if (e != cudaSuccess) break;
        // the op
        if ((e = cudaStreamWaitEvent(io.s_op, io.in_done[k], 0)) != cudaSuccess) break;
        credit_args a = blk;
        a.in = io.in_buf[k];
        a.out = io.out_buf[k];
        a.rows = n;
        if (blk.in_scale) a.in_scale = io.isc[k];
        if (blk.out_scale) a.out_scale = io.osc[k];
        if ((st = run_with_plan(dev, &a, &chosen, io.s_op)) != CREDIT_OK) {
            cudaStreamSynchronize(io.s_in);
            cudaStreamSynchronize(io.s_op);
            cudaStreamSynchronize(io.s_out);
            return st;
        }
        if ((e = cudaEventRecord(io.op_done[k], io.s_op)) != cudaSuccess) break;
        // copy-out
        if ((e = cudaStreamWaitEvent(io.s_out, io.op_done[k], 0)) != cudaSuccess) break;
        if (lse && dout)
            e = launch_copy(io.out_buf[k], n * 4, dout + r0 * 4, n * 4, 1, n * 4, io.s_out);
        else if (dout)
            e = launch_copy(io.out_buf[k], row_out, dout + r0 * ld_out * osz, ld_out * osz, n, row_out, io.s_out);
        else if (lse)
            e = cudaMemcpyAsync(hout + r0 * 4, io.out_buf[k], n * 4, cudaMemcpyDeviceToHost, io.s_out);
        else if (ld_out * osz == row_out)
            e = cudaMemcpyAsync(hout + r0 * row_out, io.out_buf[k], n * row_out, cudaMemcpyDeviceToHost, io.s_out);
        else
            e = cudaMemcpy2DAsync(hout + r0 * ld_out * osz, ld_out * osz, io.out_buf[k], row_out, row_out, n,
                                  cudaMemcpyDeviceToHost, io.s_out);
        if (e == cudaSuccess && blk.out_scale)
            e = cudaMemcpyAsync(args->out_scale + r0, io.osc[k], n * 4, cudaMemcpyDeviceToHost, io.s_out);
        if (e == cudaSuccess) e = cudaEventRecord(io.out_done[k], io.s_out);
    }
    const cudaError_t e1 = cudaStreamSynchronize(io.s_in);
    const cudaError_t e2 = cudaStreamSynchronize(io.s_op);
    const cudaError_t e3 = cudaStreamSynchronize(io.s_out);
    if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3);
    return status_of(e);
}
