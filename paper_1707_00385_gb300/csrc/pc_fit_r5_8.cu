// Instantiations of the fused kernels for window radii 5..8 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r5_8(int r) {
    static const KernelOps k5 = {launch_fit_rw<5>, launch_batch_rw<5>, occupancy_rw<5>};
    static const KernelOps k6 = {launch_fit_rw<6>, launch_batch_rw<6>, occupancy_rw<6>};
    static const KernelOps k7 = {launch_fit_rw<7>, launch_batch_rw<7>, occupancy_rw<7>};
    static const KernelOps k8 = {launch_fit_rw<8>, launch_batch_rw<8>, occupancy_rw<8>};
    switch (r) {
        case 5: return &k5;
        case 6: return &k6;
        case 7: return &k7;
        case 8: return &k8;
        default: return nullptr;
    }
}

}  // namespace pcurv
