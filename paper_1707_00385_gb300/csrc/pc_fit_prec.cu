// Instantiations of the precision variants (run-time radius and stride):
// compensated moment sums, and ranges stored as FP16/BF16 offsets from a
// per-tile FP32 base.  The batch kernel is instantiated for float32 ranges only.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_precision(int kahan, int format) {
    static const KernelOps k[6] = {
        {launch_fit_rw<0, 0>, launch_batch_rw<0, 0>, occupancy_rw<0, 0>},
        {launch_fit_rw<0, 1>, launch_batch_rw<0, 1>, occupancy_rw<0, 1>},
        {launch_fit_rw<0, 2>, nullptr, nullptr},
        {launch_fit_rw<0, 3>, nullptr, nullptr},
        {launch_fit_rw<0, 4>, nullptr, nullptr},
        {launch_fit_rw<0, 5>, nullptr, nullptr},
    };
    if (format < 0 || format > 2 || (kahan != 0 && kahan != 1)) return nullptr;
    return &k[format * 2 + kahan];
}

}  // namespace pcurv
