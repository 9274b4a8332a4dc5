// Instantiations of the fused kernels for window radii 1..4 (dense window),
// both one-lane tile variants.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r1_4(int r) {
    switch (r) {
        case 1: return make_ops<1, 0>();
        case 2: return make_ops<2, 0>();
        case 3: return make_ops<3, 0>();
        case 4: return make_ops<4, 0>();
        default: return nullptr;
    }
}

}  // namespace pcurv
