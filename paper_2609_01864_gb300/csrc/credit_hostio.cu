// credit_hostio.cu -- credit_run_host: one op on host buffers, with the rows
// streamed through device staging buffers.
//
// The rows are cut into blocks; block b's input is copied in on the h2d
// stream, the op runs on the compute stream, and the output is copied out on
// the d2h stream.  kBlocks staging slots rotate, so the copy-in of block
// b + 1, the op on block b and the copy-out of block b - 1 run at the same
// time (the host link is full duplex; the op itself takes a few percent of
// the copy time).  Events order the three streams:
//   copy-in b     waits for copy-out b - kBlocks (its slot is free again)
//   op b          waits for copy-in b
//   copy-out b    waits for op b
// The staging slots are allocated on first use and kept per device (grown
// when a larger block is needed), like the two-pass workspace.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/credit.h"
#include "credit_host.h"

namespace credit {
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
    cudaError_t e = cudaSuccess;
    long long b = 0;
    for (long long r0 = 0; r0 < rows && e == cudaSuccess; r0 += br, ++b) {
        const int k = static_cast<int>(b % kBlocks);
        const long long n = rows - r0 < br ? rows - r0 : br;
        // copy-in (slot k free once its previous copy-out finished)
        if (b >= kBlocks && (e = cudaStreamWaitEvent(io.s_in, io.out_done[k], 0)) != cudaSuccess) break;
        if (ld_in * isz == row_in)  // contiguous rows: one plain copy
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
        if (lse)
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
