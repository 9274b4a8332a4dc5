// Instantiations of the fused kernels for window radii 9..12 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r9_12(int r) {
    static const KernelOps k9 = {launch_fit_rw<9>, launch_batch_rw<9>, occupancy_rw<9>};
    static const KernelOps k10 = {launch_fit_rw<10>, launch_batch_rw<10>, occupancy_rw<10>};
    static const KernelOps k11 = {launch_fit_rw<11>, launch_batch_rw<11>, occupancy_rw<11>};
    static const KernelOps k12 = {launch_fit_rw<12>, launch_batch_rw<12>, occupancy_rw<12>};
    switch (r) {
        case 9: return &k9;
        case 10: return &k10;
        case 11: return &k11;
        case 12: return &k12;
        default: return nullptr;
    }
}

}  // namespace pcurv
