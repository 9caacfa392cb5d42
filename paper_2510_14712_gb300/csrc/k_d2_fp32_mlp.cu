// Fused step with the learned closure: D = 2, storage float, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
void step_d2_fp32_mlp(Handle& h, const void* src, void* dst) {
  OpsImpl<2, float, float>::step_cl<MlpClosure>(h, src, dst);
}
int autotune_d2_fp32_mlp(Handle& h, int reps, float* best_ms) {
  return OpsImpl<2, float, float>::autotune_cl<MlpClosure>(h, reps, best_ms);
}
int ntiles_d2_fp32_mlp() { return OpsImpl<2, float, float>::ntiles_cl<MlpClosure>(); }
}  // namespace lbm
