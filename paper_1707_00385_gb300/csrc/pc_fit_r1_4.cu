// Instantiations of the fused kernels for window radii 1..4 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r1_4(int r) {
    static const KernelOps k1 = {launch_fit_rw<1>, launch_batch_rw<1>, occupancy_rw<1>};
    static const KernelOps k2 = {launch_fit_rw<2>, launch_batch_rw<2>, occupancy_rw<2>};
    static const KernelOps k3 = {launch_fit_rw<3>, launch_batch_rw<3>, occupancy_rw<3>};
    static const KernelOps k4 = {launch_fit_rw<4>, launch_batch_rw<4>, occupancy_rw<4>};
    switch (r) {
        case 1: return &k1;
        case 2: return &k2;
        case 3: return &k3;
        case 4: return &k4;
        default: return nullptr;
    }
}

}  // namespace pcurv
