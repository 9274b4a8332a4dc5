// Instantiations of the fused kernel for window radii 1..4 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

cudaError_t launch_fit_r1_4(const float* depth, int H, int W, const Camera& cam,
                            const FitConfig& cfg, float* k1, float* k2, float* normal,
                            cudaStream_t stream) {
    switch (cfg.r) {
        case 1: return launch_fit_rw<1>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 2: return launch_fit_rw<2>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 3: return launch_fit_rw<3>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 4: return launch_fit_rw<4>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcurv
