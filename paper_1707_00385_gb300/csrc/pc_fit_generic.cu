// The fused kernel with the window radius and sampling stride read at run
// time (radii above the unrolled set, and sparse windows).
#include "pc_fit.cuh"

namespace pcurv {

cudaError_t launch_fit_generic(const float* depth, int H, int W, const Camera& cam,
                               const FitConfig& cfg, float* k1, float* k2, float* normal,
                               cudaStream_t stream) {
    return launch_fit_rw<0>(depth, H, W, cam, cfg, k1, k2, normal, stream);
}

}  // namespace pcurv
