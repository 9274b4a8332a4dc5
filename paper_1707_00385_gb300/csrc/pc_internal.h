// pc_internal.h -- what the host runtime (pc_api.cu) and the kernels
// (pc_fit_*.cu) share.  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

namespace pcurv {

// Pinhole intrinsics (pixels) and their reciprocals.
struct Camera {
    float fx, fy, cx, cy;
    float ifx, ify;
};

// Method parameters as the kernels read them.
struct FitConfig {
    int r;             // window radius
    int rn;            // initial-normal radius
    int T;             // re-weighted iterations
    int stride;        // window sampling stride
    float invk;        // 1/k of W(eps) = k/(k+eps^2) = 1/(1 + eps^2/k)
    int reject;        // rejection filter on/off
    float reject_ratio;
    float det_tol;
    float pivot_tol;
    int min_window;
};

// Output tile of one CTA: TILE_W x TILE_H pixels, one thread per pixel.
constexpr int TILE_W = 32;
constexpr int TILE_H = 8;
constexpr int BLOCK_THREADS = TILE_W * TILE_H;

inline int halo_of(const FitConfig& c) { return c.r > c.rn ? c.r : c.rn; }

// Z and c planes of the tile + halo, and per-row valid counts.
inline size_t fit_smem_bytes(const FitConfig& c) {
    const int h = halo_of(c);
    return (size_t)(TILE_W + 2 * h) * (TILE_H + 2 * h) * 2 * sizeof(float) +
           (size_t)(TILE_H + 2 * h) * TILE_W * sizeof(int);
}

// Enqueues the fused per-pixel kernel for one H x W image on `stream`.
// normal may be nullptr.  Returns the launch error (cudaSuccess on success).
cudaError_t launch_fit(const float* depth, int H, int W, const Camera& cam, const FitConfig& cfg,
                       float* k1, float* k2, float* normal, cudaStream_t stream);

// Instantiation groups (one translation unit each, compiled in parallel).
cudaError_t launch_fit_r1_4(const float*, int, int, const Camera&, const FitConfig&, float*, float*,
                            float*, cudaStream_t);
cudaError_t launch_fit_r5_8(const float*, int, int, const Camera&, const FitConfig&, float*, float*,
                            float*, cudaStream_t);
cudaError_t launch_fit_r9_12(const float*, int, int, const Camera&, const FitConfig&, float*, float*,
                             float*, cudaStream_t);
cudaError_t launch_fit_generic(const float*, int, int, const Camera&, const FitConfig&, float*,
                               float*, float*, cudaStream_t);

}  // namespace pcurv
