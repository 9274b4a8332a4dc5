// Instantiations of the fused kernel for window radii 5..8 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

cudaError_t launch_fit_r5_8(const float* depth, int H, int W, const Camera& cam,
                            const FitConfig& cfg, float* k1, float* k2, float* normal,
                            cudaStream_t stream) {
    switch (cfg.r) {
        case 5: return launch_fit_rw<5>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 6: return launch_fit_rw<6>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 7: return launch_fit_rw<7>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 8: return launch_fit_rw<8>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcurv
