// pc_outputs.cu -- organised outputs for downstream use: the point cloud of
// the back-projection (Sec. 3.2, first item) and the field of initial normals
// (Sec. 3.2.1, Eq. initialnormal) on their own, without the quadric fit.
//
// k_backproject is a stream over the image (4 B in, 12 B out per pixel):
// each thread converts four consecutive pixels, with 16-byte loads and stores
// when the buffers allow.  k_initial_normals stages a 32 x (8 PPT) tile plus a halo
// of rn pixels in shared memory and runs the same regression device function
// as the full path, so its normals equal those pc_compute starts from.
#include <cfloat>
#include <cstdint>

#include "pc_fit.cuh"

namespace pcurv {

namespace {

__device__ __forceinline__ bool range_ok(float z) { return z > 0.f && z <= FLT_MAX; }

// ((u - cx) z / fx, (v - cy) z / fy, z), NaN for a pixel without a valid range.
// Correctly rounded division keeps each coordinate within 1.5 ulp of the exact value.
__device__ __forceinline__ float3 point_of(float z, int u, int v, const Camera& cam) {
    if (!range_ok(z)) {
        const float q = __int_as_float(0x7fffffff);
        return make_float3(q, q, q);
    }
    return make_float3(__fdiv_rn(((float)u - cam.cx) * z, cam.fx), __fdiv_rn(((float)v - cam.cy) * z, cam.fy), z);
}

constexpr int BP_THREADS = 256;
constexpr int BP_WARPS = BP_THREADS / 32;
constexpr int BP_BLOCKS_PER_SM = 8;  // 64 resident warps per SM: the whole grid is one wave

// VEC: depth and xyz are 16-byte aligned and W is a multiple of 4, so that a
// group of four pixels is one float4 of ranges and three float4 of points and
// lies in one row.  A warp takes 32 consecutive groups (128 pixels): one
// coalesced 512-byte load, then its 96 float4 of points go through shared
// memory so that each of the three stores writes 512 contiguous bytes (lane l
// stages float4 3l .. 3l+2: a quarter warp covers 8 disjoint 4-bank groups,
// free of bank conflicts).  H * W < 2^31 (PC_MAX_DIM^2): 32-bit indices.
template <bool VEC>
__global__ void __launch_bounds__(BP_THREADS, BP_BLOCKS_PER_SM)
    k_backproject(const float* __restrict__ depth, int H, int W, Camera cam, float* __restrict__ xyz) {
    const unsigned n = (unsigned)H * (unsigned)W;
    const unsigned groups = (n + 3) / 4;
    const unsigned uw = (unsigned)W;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (VEC) {
        __shared__ float4 stage[BP_WARPS][96];
        float4* st = stage[warp];
        const unsigned nwarps = gridDim.x * BP_WARPS;
        for (unsigned w0 = (blockIdx.x * BP_WARPS + warp) * 32; w0 < groups; w0 += nwarps * 32) {
            const unsigned g = w0 + lane;
            if (g < groups) {
                const float4 z = __ldcs(reinterpret_cast<const float4*>(depth) + g);
                const unsigned v = 4 * g / uw, u = 4 * g - v * uw;
                const float3 p0 = point_of(z.x, (int)u, (int)v, cam), p1 = point_of(z.y, (int)u + 1, (int)v, cam),
                             p2 = point_of(z.z, (int)u + 2, (int)v, cam), p3 = point_of(z.w, (int)u + 3, (int)v, cam);
                st[3 * lane] = make_float4(p0.x, p0.y, p0.z, p1.x);
                st[3 * lane + 1] = make_float4(p1.y, p1.z, p2.x, p2.y);
                st[3 * lane + 2] = make_float4(p2.z, p3.x, p3.y, p3.z);
            }
            __syncwarp();
            const unsigned live = 3 * min(32u, groups - w0);   // float4 of points this warp writes
            float4* o = reinterpret_cast<float4*>(xyz) + 3 * (size_t)w0;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const unsigned k = 32 * j + lane;
                if (k < live) __stcs(o + k, st[k]);  // streaming: written once, not read back here
            }
            __syncwarp();
        }
    } else {
        const unsigned stride = gridDim.x * BP_THREADS;
        for (unsigned g = blockIdx.x * BP_THREADS + threadIdx.x; g < groups; g += stride) {
            for (unsigned i = 4 * g; i < 4 * g + 4 && i < n; i++) {
                const unsigned v = i / uw, u = i - v * uw;
                const float3 p = point_of(depth[i], (int)u, (int)v, cam);
                xyz[3 * (size_t)i] = p.x;
                xyz[3 * (size_t)i + 1] = p.y;
                xyz[3 * (size_t)i + 2] = p.z;
            }
        }
    }
}

// One CTA per 32 x (TH PPT) output tile: each thread computes PPT pixels of
// its column, TH rows apart, so that one staging of the tile's Z plane plus a
// halo of rn (0 where the range is not valid, as the full path stages it)
// serves PPT times the arithmetic.  Registers are bounded for four 256-thread
// CTAs per SM (the 7x7 patch, unrolled, would otherwise take more and leave
// three).
template <int TH, int PPT>
__global__ void __launch_bounds__(TILE_W * TH, 4 * 8 / TH)
    k_initial_normals(const float* __restrict__ depth, int H, int W, Camera cam, int rn, float det_tol,
                      float* __restrict__ normal) {
    extern __shared__ float smem[];
    constexpr int NT = TILE_W * TH;
    constexpr int TROWS = TH * PPT;
    const int SW = TILE_W + 2 * rn, SH = TROWS + 2 * rn;
    float* tz = smem;
    const int ub = blockIdx.x * TILE_W, vb = blockIdx.y * TROWS;
    const int tid = threadIdx.y * TILE_W + threadIdx.x;
    // element i = sy SW + sx, advanced by NT per step without a division
    const int dy = NT / SW, dx = NT - dy * SW;
    int sy = tid / SW, sx = tid - sy * SW;
    for (int i = tid; i < SW * SH; i += NT) {
        const int gv = vb - rn + sy, gu = ub - rn + sx;
        float z = 0.f;
        if (gu >= 0 && gu < W && gv >= 0 && gv < H) {
            const float d = __ldg(depth + (size_t)gv * W + gu);
            if (range_ok(d)) z = d;
        }
        tz[i] = z;
        sx += dx;
        sy += dy;
        if (sx >= SW) {
            sx -= SW;
            sy++;
        }
    }
    __syncthreads();
    const int u0 = ub + threadIdx.x;
    if (u0 >= W) return;
#pragma unroll 1
    for (int k = 0; k < PPT; k++) {
        const int row = threadIdx.y + k * TH;
        const int v0 = vb + row;
        if (v0 >= H) return;
        const int cidx = (row + rn) * SW + threadIdx.x + rn;
        const float Zp = tz[cidx];
        float nx = 0.f, ny = 0.f, nz = 1.f;
        bool ok = Zp > 0.f;
        if (ok)
            ok = rn == NORMAL_RADIUS_UNROLLED
                     ? initial_normal<NORMAL_RADIUS_UNROLLED, true>(tz + cidx, SW, 0, (float)u0 - cam.cx,
                                                                    (float)v0 - cam.cy, Zp, cam, det_tol, nx, ny,
                                                                    nz)
                     : initial_normal<0>(tz + cidx, SW, rn, (float)u0 - cam.cx, (float)v0 - cam.cy, Zp, cam,
                                         det_tol, nx, ny, nz);
        const size_t out = (size_t)v0 * W + u0;
        const float q = __int_as_float(0x7fffffff);
        normal[3 * out] = ok ? nx : q;
        normal[3 * out + 1] = ok ? ny : q;
        normal[3 * out + 2] = ok ? nz : q;
    }
}

constexpr int NORMAL_TH = 8;
constexpr int NORMAL_BLOCKS_PER_SM = 4;  // the kernel's launch bound

}  // namespace

cudaError_t launch_backproject(const float* depth, int H, int W, const Camera& cam, float* xyz, int sms,
                               cudaStream_t stream) {
    const size_t groups = ((size_t)H * W + 3) / 4;
    const size_t want = (groups + BP_THREADS - 1) / BP_THREADS;
    const size_t cap = (size_t)(sms > 0 ? sms : 152) * BP_BLOCKS_PER_SM;
    const int grid = (int)(want < cap ? want : cap);
    const bool vec = ((uintptr_t)depth & 15u) == 0 && ((uintptr_t)xyz & 15u) == 0 && (W & 3) == 0;
    if (vec)
        k_backproject<true><<<grid, BP_THREADS, 0, stream>>>(depth, H, W, cam, xyz);
    else
        k_backproject<false><<<grid, BP_THREADS, 0, stream>>>(depth, H, W, cam, xyz);
    return cudaGetLastError();
}

// Pixels per thread: each thread computes PPT pixels of its column from one
// staged 32 x (8 PPT) tile plus halo, so the tile's global loads and barrier
// wait are spread over PPT times the arithmetic.  GB300, one 4096 x 4096 image
// (same bits): 0.508 ms with one pixel per thread, 0.464 with two, 0.442 with
// four, 0.430 with eight.  Taller tiles make a smaller grid, so the launch
// takes the largest PPT that still gives at least two waves of CTAs (a 640 x
// 480 frame keeps one pixel per thread).
static size_t initial_normals_smem_bytes(int rn, int ppt) {
    return (size_t)(TILE_W + 2 * rn) * (NORMAL_TH * ppt + 2 * rn) * sizeof(float);
}

template <int PPT>
static cudaError_t launch_normals_ppt(const float* depth, int H, int W, const Camera& cam, int rn, float det_tol,
                                      float* normal, cudaStream_t stream) {
    constexpr int rows = NORMAL_TH * PPT;
    const dim3 block(TILE_W, NORMAL_TH);
    const dim3 grid((W + TILE_W - 1) / TILE_W, (H + rows - 1) / rows);
    k_initial_normals<NORMAL_TH, PPT>
        <<<grid, block, initial_normals_smem_bytes(rn, PPT), stream>>>(depth, H, W, cam, rn, det_tol, normal);
    return cudaGetLastError();
}

cudaError_t launch_initial_normals(const float* depth, int H, int W, const Camera& cam, int rn, float det_tol,
                                   float* normal, int sms, cudaStream_t stream) {
    const long long wave = 2LL * NORMAL_BLOCKS_PER_SM * (sms > 0 ? sms : 152);
    const long long cols = (W + TILE_W - 1) / TILE_W;
    auto tiles = [&](int ppt) { return cols * ((H + NORMAL_TH * ppt - 1) / (NORMAL_TH * ppt)); };
    if (tiles(8) >= wave) return launch_normals_ppt<8>(depth, H, W, cam, rn, det_tol, normal, stream);
    if (tiles(4) >= wave) return launch_normals_ppt<4>(depth, H, W, cam, rn, det_tol, normal, stream);
    if (tiles(2) >= wave) return launch_normals_ppt<2>(depth, H, W, cam, rn, det_tol, normal, stream);
    return launch_normals_ppt<1>(depth, H, W, cam, rn, det_tol, normal, stream);
}

}  // namespace pcurv
