// credit_model.h -- cost models used by the planner (internal).
#pragma once

#include "credit_host.h"

namespace credit {

// Fill *p from the loaded calibration / learned model.  Returns false when no
// model is loaded (the caller then uses the built-in heuristic).
bool model_plan(const DeviceInfo &di, int device, int op, long long rows, long long cols, int tin, int tout,
                credit_plan_t *p);

}  // namespace credit
