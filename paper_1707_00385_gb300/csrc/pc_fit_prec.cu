// Instantiations of the precision variants (run-time radius and stride,
// 32 x 8 tiles): compensated moment sums, and ranges stored as FP16/BF16
// offsets from a per-tile base.  The batch kernel is instantiated for
// float32 ranges only.
#include "pc_fit.cuh"

namespace pcurv {

const KernelOps* ops_precision(int kahan, int format) {
    static const KernelOps k[6] = {
        {{launch_fit_rw<0, 0, 8>, nullptr}, {launch_batch_rw<0, 0, 8>, nullptr}, {occupancy_rw<0, 0, 8>, nullptr}},
        {{launch_fit_rw<0, 1, 8>, nullptr}, {launch_batch_rw<0, 1, 8>, nullptr}, {occupancy_rw<0, 1, 8>, nullptr}},
        {{launch_fit_rw<0, 2, 8>, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}},
        {{launch_fit_rw<0, 3, 8>, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}},
        {{launch_fit_rw<0, 4, 8>, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}},
        {{launch_fit_rw<0, 5, 8>, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}},
    };
    if (format < 0 || format > 2 || (kahan != 0 && kahan != 1)) return nullptr;
    return &k[format * 2 + kahan];
}

}  // namespace pcurv
