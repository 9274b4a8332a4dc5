// Instantiations of the precision variants (run-time radius and stride,
// 32 x 8 tiles, per-frame and persistent batch kernels): compensated moment
// sums, and ranges stored as FP16/BF16 offsets from a per-tile base.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_precision(int kahan, int format) {
#define PC_PREC_OPS(P) {{launch_fit_rw<0, P, 8>, nullptr}, {launch_batch_rw<0, P, 8>, nullptr}, {occupancy_rw<0, P, 8>, nullptr}}
    static const KernelOps k[6] = {PC_PREC_OPS(0), PC_PREC_OPS(1), PC_PREC_OPS(2),
                                   PC_PREC_OPS(3), PC_PREC_OPS(4), PC_PREC_OPS(5)};
#undef PC_PREC_OPS
    if (format < 0 || format > 2 || (kahan != 0 && kahan != 1)) return nullptr;
    return &k[format * 2 + kahan];
}

}  // namespace pcurv
