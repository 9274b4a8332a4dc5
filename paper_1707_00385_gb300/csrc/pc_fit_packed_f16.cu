// Instantiations for ranges stored as FP16 offsets from a per-tile base,
// with the window columns unrolled for the radii the precision sweep uses
// (3, 7 and 11; dense windows, plain sums), both one-lane tile variants.
// Other radii, strides and compensated sums take the run-time-radius kernels
// of pc_fit_prec.cu.  The arithmetic after loading a range is the float32
// kernels' own.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_packed_f16(int r) {
    switch (r) {
        case 3: return make_ops<3, 2>();
        case 7: return make_ops<7, 2>();
        case 11: return make_ops<11, 2>();
        default: return nullptr;
    }
}

}  // namespace pcurv
