// Kernel set: D = 2, storage double, arithmetic double.
#include "lbm_ops.cuh"

namespace lbm {
const Ops* ops_d2_fp64() { return OpsImpl<2, double, double>::ops(); }
size_t scratch_bytes_d2_fp64(const Params& p) { return OpsImpl<2, double, double>::scratch_bytes(p); }
}  // namespace lbm
