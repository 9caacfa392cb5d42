// Kernel set: D = 2, storage float, arithmetic float.
#include "lbm_ops.cuh"

namespace lbm {
const Ops* ops_d2_fp32() { return OpsImpl<2, float, float>::ops(); }
size_t scratch_bytes_d2_fp32(const Params& p) { return OpsImpl<2, float, float>::scratch_bytes(p); }
}  // namespace lbm
