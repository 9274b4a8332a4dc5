// Instantiations of the fused kernels for window radii 9..12 (dense window),
// both one-lane tile variants.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_r9_12(int r) {
    switch (r) {
        case 9: return make_ops<9, 0>();
        case 10: return make_ops<10, 0>();
        case 11: return make_ops<11, 0>();
        case 12: return make_ops<12, 0>();
        default: return nullptr;
    }
}

}  // namespace pcurv
