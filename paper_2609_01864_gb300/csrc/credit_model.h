// credit_model.h -- cost models used by the planner (internal).
#pragma once

#include "credit_host.h"

namespace credit {

// Fill *p from the loaded calibration (analytic model, or the learned model
// when CREDIT_MODEL=learned).  Returns false when no calibration is loaded
// (the caller then uses the built-in heuristic).
bool model_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                credit_plan_t *p);

// Analytic model (Eq. 7-9; ablation = 1: Table IV's peak-bandwidth +
// serialized-staging model).  best_dT receives the winning dT (us).
bool analytic_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                   int ablation, credit_plan_t *p, double *best_dT);

// Learned model: argmin of the predicted latency over the legal candidates.
bool learned_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                  credit_plan_t *p);
// The same, restricted to the non-cluster candidates.
bool learned_plan_no_cluster(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin,
                             int tout, credit_plan_t *p);

int two_pass_split(int sm_count, long long rows, long long cols, int isz);

// The selected non-DSMEM baseline plan of a shape (Sec. IV-A) and its time
// T_B (us) from the loaded calibration (Eq. 7's measured baseline timing,
// interpolated over the calibration grid).  false (T_B = 0) without one.
bool baseline_estimate(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                       credit_plan_t *base, double *T_B_us);

}  // namespace credit

extern "C" credit_status credit_mlp_load(const char *path);
