// Fused step with the FP64 temperature inversion (exact van der Waals
// closure): D = 3, storage float, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
void step_d3_fp32_t64(Handle& h, const void* src, void* dst) {
  OpsImpl<3, float, float>::step_cl<ExactClosure<float, true>>(h, src, dst);
}
int autotune_d3_fp32_t64(Handle& h, int reps, float* best_ms) {
  return OpsImpl<3, float, float>::autotune_cl<ExactClosure<float, true>>(h, reps, best_ms);
}
int ntiles_d3_fp32_t64() { return OpsImpl<3, float, float>::ntiles_cl<ExactClosure<float, true>>(); }
}  // namespace lbm
