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
    int kahan;         // compensated moment sums
    float fp64_pivot;  // refactorise in FP64 below this scaled pivot (0 = never)
};

// Output tile of one CTA: TILE_W x th pixels, in five variants
//   0: 32 x 8 pixels, one thread each (256 threads)
//   1: 32 x 4 pixels, one thread each (128 threads; frames with few tiles)
//   2: 32 x 4 pixels, 2 lanes each; 3: 32 x 2, 4 lanes; 4: 32 x 1, 8 lanes
//      (256 threads; the lanes of a pixel share its window rows)
// Variants 0 and 1 give the same bits; the lane groups add the moment sums in
// another order, which changes single-precision rounding only.
constexpr int TILE_W = 32;
constexpr int NUM_TILE_VARIANTS = 5;
inline int tile_h_of(int variant) {
    constexpr int h[NUM_TILE_VARIANTS] = {8, 4, 4, 2, 1};
    return h[variant];
}
inline int lanes_of(int variant) {
    constexpr int g[NUM_TILE_VARIANTS] = {1, 1, 2, 4, 8};
    return g[variant];
}
// The variant of a lane-group size (2, 4, 8), else -1.
inline int variant_of_lanes(int lanes) { return lanes == 2 ? 2 : lanes == 4 ? 3 : lanes == 8 ? 4 : -1; }
// storage tiles of the 16-bit range format (pc_pack_depth): 32 x 8
constexpr int PACK_TILE_H = 8;

// The initial-normal patch radius compiled with unrolled loops: 3, the 7 x 7
// patch of Sec. 3.2.1 (other radii run the same code with run-time loops).
constexpr int NORMAL_RADIUS_UNROLLED = 3;

inline int halo_of(const FitConfig& c) { return c.r > c.rn ? c.r : c.rn; }

// Sums of J^T W J whose running totals the one-lane FP32 kernels keep in
// shared memory, as one pair of floats per thread (fit_tile, fold_rows).
constexpr int FOLD_SUMS = 20;

// Z and c planes of the tile + halo, per-row valid counts and, for
// fold_threads > 0, the folded totals of that many threads (8-byte aligned).
inline size_t fit_smem_bytes(const FitConfig& c, int th, int fold_threads = 0) {
    const int h = halo_of(c);
    const size_t planes = (size_t)(TILE_W + 2 * h) * (th + 2 * h) * 2 * sizeof(float) +
                          (size_t)(th + 2 * h) * TILE_W * sizeof(int);
    return (planes + 7) / 8 * 8 + (size_t)fold_threads * FOLD_SUMS * 8;
}

inline long long tiles_of(int H, int W, int th) {
    return (long long)((W + TILE_W - 1) / TILE_W) * ((H + th - 1) / th);
}

// One frame: caller-owned device buffers, size and intrinsics.
struct FrameArgs {
    const float* depth;
    int H, W;
    Camera cam;
    float* k1;
    float* k2;
    float* normal;  // may be nullptr
    // centred 16-bit storage instead of depth (precision variants): per pixel
    // an offset, per 32x8 tile an FP32 base
    const unsigned short* packed;
    const float* tile_base;
};

// A frame of a batch and its place in the flattened tile queue.
struct BatchFrame {
    FrameArgs f;
    int tiles_x;     // tiles per row of this frame
    int tile_begin;  // first queue index of this frame
};

// Device-resident batch table: header followed by nframes descriptors.
struct BatchTable {
    int nframes;
    int total_tiles;
    int pad[2];
    BatchFrame frames[1];  // nframes entries
};

inline size_t batch_table_bytes(int nframes) {
    return sizeof(BatchTable) + (size_t)(nframes > 1 ? nframes - 1 : 0) * sizeof(BatchFrame);
}

// Kernel entry points of one instantiation (window radius, dense or run-time),
// per tile variant (nullptr where a variant is not compiled).
struct KernelOps {
    // tile rows [ty0, ty1) of one frame (the variant's tile height)
    cudaError_t (*fit[NUM_TILE_VARIANTS])(const FrameArgs&, const FitConfig&, cudaStream_t, int ty0, int ty1);
    cudaError_t (*batch[NUM_TILE_VARIANTS])(const BatchTable*, unsigned*, int, const FitConfig&, cudaStream_t);
    cudaError_t (*occupancy[NUM_TILE_VARIANTS])(const FitConfig&, int*);
};

// Instantiation groups (one translation unit each, compiled in parallel);
// each returns its table for radius r, or nullptr.  ops_r* and ops_generic
// hold the one-lane variants, ops_lanes the lane-group variants (run-time
// radius and stride, serving every window).
const KernelOps* ops_r1_4(int r);
const KernelOps* ops_r5_8(int r);
const KernelOps* ops_r9_12(int r);
const KernelOps* ops_generic();
const KernelOps* ops_lanes();
// The sparsely sampled 37 x 37 patch of Sec. 4.2.1 (radius 18, read as every
// third pixel), unrolled like the dense radii; nullptr for other windows.
constexpr int SPARSE_RADIUS = 18, SPARSE_STRIDE = 3;
const KernelOps* ops_sparse(int r, int stride);

// Run-time-radius kernels of the precision variants: compensated sums and/or
// 16-bit range storage (format 0 float32, 1 FP16, 2 BF16).
const KernelOps* ops_precision(int kahan, int format);
// 16-bit range storage with unrolled columns for window radii 3, 7 and 11
// (plain sums), else nullptr.
const KernelOps* ops_packed_f16(int r);
const KernelOps* ops_packed_bf16(int r);
// The kernels reading 16-bit storage of `format` (1 FP16, 2 BF16) under cfg.
const KernelOps* select_packed_ops(const FitConfig& cfg, int format);

// The instantiation serving cfg (dense radii 1..12 unrolled, anything else
// run-time; compensated sums on the precision kernels), all five variants.
const KernelOps* select_ops(const FitConfig& cfg);

// Packs float32 ranges into per-tile-centred 16-bit storage (format 1 FP16, 2 BF16).
cudaError_t launch_pack(const float* depth, int H, int W, int format, unsigned short* packed,
                        float* tile_base, cudaStream_t stream);

// Organised outputs (pc_outputs.cu): point cloud and initial-normal field.
cudaError_t launch_backproject(const float* depth, int H, int W, const Camera& cam, float* xyz, int sms,
                               cudaStream_t stream);
cudaError_t launch_initial_normals(const float* depth, int H, int W, const Camera& cam, int rn, float det_tol,
                                   float* normal, int sms, cudaStream_t stream);

}  // namespace pcurv

struct pc_ctx;

namespace pcurv {

// Read access to a context's kernel parameters, and a way to leave a message
// for pc_last_error(), for entry points defined outside pc_api.cu.
const FitConfig& ctx_config(const pc_ctx* ctx);
void ctx_set_error(pc_ctx* ctx, const char* msg);
// The tile variant the context's parameters force (a lane group of
// lanes_per_pixel, or a one-lane tile height), else -1.
int ctx_forced_variant(const pc_ctx* ctx);

}  // namespace pcurv
