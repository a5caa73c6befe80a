// credit_host.h -- internal host-side declarations shared by the library's
// translation units (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/credit.h"

namespace credit {

struct DeviceInfo {
    int sm_count;
    long long smem_optin;     // max dynamic shared memory per block (opt-in)
    long long smem_per_sm;
    int cc_major, cc_minor;
    int clock_khz;
    size_t ws_floats;         // two-pass workspace capacity in floats
};

int dtype_size(int dt);
int current_device();
const DeviceInfo *device_info(int device);
// Staged-path (ring kernel) geometry for one shape and cluster size.
struct RingCfg {
    int P;
    int chunk;           // bytes per chunk
    int ring;            // chunk slots
    int threads;         // reducer + writer threads + one producer warp
    int reducers;        // reducer threads
    int affine;          // gamma/beta ring slots (0: direct loads)
    int affine_resident; // slots hold the whole slice's gamma/beta
    long long aslot;     // bytes per affine slot
    long long smem;      // dynamic shared memory per CTA
    long long body_max;  // largest slice body (bytes) of any CTA
    int nch_max;         // chunks of the largest slice
    int tmem;            // 1: the slice is retained in tensor memory (k_ring_tm)
};
// nab: gamma/beta arrays streamed through the affine ring (0, 1 or 2).
bool ring_config(const DeviceInfo &di, long long N, int isz, int P, int req_ring, int req_chunk, int req_threads,
                 int req_reducers, int nab, RingCfg *out);
// Slices above this many bytes are retained in tensor memory when a plan
// leaves the tier to the library (AUTO): below it the shared-memory ring fits
// several CTAs per SM.
constexpr long long kTmAutoMinSlice = 32768;
// Tensor-memory retention geometry (k_ring_tm); false where it does not apply.
bool ring_config_tm(const DeviceInfo &di, long long N, int isz, int P, int req_ring, int req_chunk, int nab,
                    RingCfg *out);
int ring_max_clusters(int device, int op, int tin, int tout, int P, int threads, long long smem, bool tm = false);
int affine_arrays(const credit_args *a);
int affine_arrays_aligned(const credit_args *a);
extern bool g_auto_retain_tmem;
constexpr float kMaxFillShare = 0.9f;  // largest fill_share a cluster plan may carry
credit_status validate_args(const credit_args *a);
credit_status check_plan(int device, const credit_args *a, const credit_plan_t *p);
credit_status run_with_plan(int device, const credit_args *a, const credit_plan_t *p, cudaStream_t s);
credit_status ensure_init(int *device_out, cudaStream_t s);

// Shared pieces of the per-device state for the other translation units.
// Max resident clusters (CTAs when P = 1; one_per_sm: only one CTA per SM
// allowed) of a staged kernel with this launch shape; 0 if it cannot run.
int staged_max_clusters(int device, const void *fn, int P, int threads, long long smem, bool one_per_sm);
// Raise the opt-in shared memory and non-portable cluster attributes of fn once.
credit_status prepare_staged_kernel(int device, const void *fn);
unsigned *device_error_word(int device);
float *device_workspace(int device, size_t *floats);
// Launch fn with a cluster dimension of `cluster` (<= 1: no cluster attribute).
cudaError_t launch_kernel(const void *fn, dim3 grid, dim3 block, size_t smem, int cluster, cudaStream_t s,
                          void **args);

// Generation of the planner's inputs (calibration, learned model): bumped by
// every change to them, which empties the plan cache of credit_plan_ex.
void bump_plan_generation();

}  // namespace credit
