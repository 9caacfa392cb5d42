// Fused step with the FP64 temperature inversion (exact van der Waals
// closure): D = 2, storage Fp16Dev, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
void step_d2_fp16_t64(Handle& h, const void* src, void* dst) {
  OpsImpl<2, Fp16Dev, float>::step_cl<ExactClosure<float, true>>(h, src, dst);
}
int autotune_d2_fp16_t64(Handle& h, int reps, float* best_ms) {
  return OpsImpl<2, Fp16Dev, float>::autotune_cl<ExactClosure<float, true>>(h, reps, best_ms);
}
int ntiles_d2_fp16_t64() { return OpsImpl<2, Fp16Dev, float>::ntiles_cl<ExactClosure<float, true>>(); }
}  // namespace lbm
