// The fused kernels with the window radius and sampling stride read at run
// time (radii above the unrolled set, and sparse windows other than the
// 37 x 37 patch), both one-lane tile variants.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_generic() { return make_ops<0, 0>(); }

}  // namespace pcurv
