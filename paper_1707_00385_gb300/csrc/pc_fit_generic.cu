// The fused kernels with the window radius and sampling stride read at run
// time (radii above the unrolled set, and sparse windows).
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_generic() {
    static const KernelOps k = {launch_fit_rw<0>, launch_batch_rw<0>, occupancy_rw<0>};
    return &k;
}

}  // namespace pcurv
