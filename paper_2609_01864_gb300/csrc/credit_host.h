// credit_host.h -- internal host-side declarations shared by the library's
// translation units (not part of the public C ABI).
#pragma once

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
long long staged_smem_bytes(long long N, int isz, int P);
long long staged_groups_per_cta(long long N, int isz, int P);
int staged_max_clusters(int device, int op, int tin, int tout, int P, int threads, long long smem);
credit_status validate_args(const credit_args *a);
credit_status check_plan(int device, const credit_args *a, const credit_plan_t *p);
credit_status ensure_init(int *device_out, cudaStream_t s);

}  // namespace credit
