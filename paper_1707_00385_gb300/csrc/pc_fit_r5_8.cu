// Instantiations of the fused kernels for window radii 5..8 (dense window),
// both one-lane tile variants.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r5_8(int r) {
    switch (r) {
        case 5: return make_ops<5, 0>();
        case 6: return make_ops<6, 0>();
        case 7: return make_ops<7, 0>();
        case 8: return make_ops<8, 0>();
        default: return nullptr;
    }
}

}  // namespace pcurv
