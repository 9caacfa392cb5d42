// Kernel set: D = 3, storage float, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
const Ops* ops_d3_fp32() { return OpsImpl<3, float, float>::ops(); }
size_t scratch_bytes_d3_fp32(const Params& p) { return OpsImpl<3, float, float>::scratch_bytes(p); }
}  // namespace lbm
