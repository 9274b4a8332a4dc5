// Instantiations of the fused kernels with lane groups (2, 4 or 8 lanes per
// pixel), window radius and sampling stride read at run time.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_lanes() { return make_lane_ops<0>(); }

}  // namespace pcurv
