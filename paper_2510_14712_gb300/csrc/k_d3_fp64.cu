// Kernel set: D = 3, storage double, arithmetic double.
#include "lbm_ops.cuh"

namespace lbm {
const Ops* ops_d3_fp64() { return OpsImpl<3, double, double>::ops(); }
size_t scratch_bytes_d3_fp64(const Params& p) { return OpsImpl<3, double, double>::scratch_bytes(p); }
}  // namespace lbm
