// Fused step with the exact Peng-Robinson closure: D = 2, FP32 and FP64 storage
// and arithmetic, FP32 also with the FP64 temperature inversion.
#include "lbm_ops.cuh"

namespace lbm {
void step_d2_fp32_pr(Handle& h, const void* src, void* dst) {
  OpsImpl<2, float, float>::step_cl<PrClosure<float>>(h, src, dst);
}
int autotune_d2_fp32_pr(Handle& h, int reps, float* best_ms) {
  return OpsImpl<2, float, float>::autotune_cl<PrClosure<float>>(h, reps, best_ms);
}
int ntiles_d2_fp32_pr() { return OpsImpl<2, float, float>::ntiles_cl<PrClosure<float>>(); }
void step_d2_fp64_pr(Handle& h, const void* src, void* dst) {
  OpsImpl<2, double, double>::step_cl<PrClosure<double>>(h, src, dst);
}
int autotune_d2_fp64_pr(Handle& h, int reps, float* best_ms) {
  return OpsImpl<2, double, double>::autotune_cl<PrClosure<double>>(h, reps, best_ms);
}
int ntiles_d2_fp64_pr() { return OpsImpl<2, double, double>::ntiles_cl<PrClosure<double>>(); }
void step_d2_fp32_pr_t64(Handle& h, const void* src, void* dst) {
  OpsImpl<2, float, float>::step_cl<PrClosure<float, true>>(h, src, dst);
}
int autotune_d2_fp32_pr_t64(Handle& h, int reps, float* best_ms) {
  return OpsImpl<2, float, float>::autotune_cl<PrClosure<float, true>>(h, reps, best_ms);
}
int ntiles_d2_fp32_pr_t64() { return OpsImpl<2, float, float>::ntiles_cl<PrClosure<float, true>>(); }
}  // namespace lbm
