// Kernel set: D = 3, storage Fp16Dev, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
const Ops* ops_d3_fp16() { return OpsImpl<3, Fp16Dev, float>::ops(); }
size_t scratch_bytes_d3_fp16(const Params& p) { return OpsImpl<3, Fp16Dev, float>::scratch_bytes(p); }
}  // namespace lbm
