// Instantiations of the fused kernel for window radii 9..12 (dense window).
#include "pc_fit.cuh"

namespace pcurv {

cudaError_t launch_fit_r9_12(const float* depth, int H, int W, const Camera& cam,
                            const FitConfig& cfg, float* k1, float* k2, float* normal,
                            cudaStream_t stream) {
    switch (cfg.r) {
        case 9: return launch_fit_rw<9>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 10: return launch_fit_rw<10>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 11: return launch_fit_rw<11>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        case 12: return launch_fit_rw<12>(depth, H, W, cam, cfg, k1, k2, normal, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pcurv
