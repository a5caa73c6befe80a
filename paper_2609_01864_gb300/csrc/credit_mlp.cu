// credit_mlp.cu -- learned latency model (placeholder until the MLP lands).
#include "credit_model.h"

namespace credit {
bool learned_plan(const DeviceInfo &, int, int, long long, long long, int, int, credit_plan_t *) { return false; }
}  // namespace credit

extern "C" credit_status credit_mlp_load(const char *) { return CREDIT_ERR_IO; }
