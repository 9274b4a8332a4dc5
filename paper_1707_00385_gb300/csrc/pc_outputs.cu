// pc_outputs.cu -- organised outputs for downstream use: the point cloud of
// the back-projection (Sec. 3.2, first item) and the field of initial normals
// (Sec. 3.2.1, Eq. initialnormal) on their own, without the quadric fit.
//
// k_backproject is a stream over the image (4 B in, 12 B out per pixel):
// each thread converts four consecutive pixels, with 16-byte loads and stores
// when the buffers allow.  k_initial_normals stages a 32 x TH tile plus a halo
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

// VEC: depth and xyz are 16-byte aligned and W is a multiple of 4, so that a
// group of four pixels is one float4 of ranges, three float4 of points, and
// lies in one row.
template <bool VEC>
__global__ void __launch_bounds__(BP_THREADS) k_backproject(const float* __restrict__ depth, int H, int W,
                                                            Camera cam, float* __restrict__ xyz) {
    const size_t n = (size_t)H * W;
    const size_t groups = (n + 3) / 4;
    for (size_t g = (size_t)blockIdx.x * BP_THREADS + threadIdx.x; g < groups; g += (size_t)gridDim.x * BP_THREADS) {
        const size_t i0 = 4 * g;
        if (VEC) {
            const int v = (int)(i0 / (size_t)W), u = (int)(i0 - (size_t)v * W);
            const float4 z = __ldg(reinterpret_cast<const float4*>(depth) + g);
            const float3 p0 = point_of(z.x, u, v, cam), p1 = point_of(z.y, u + 1, v, cam),
                         p2 = point_of(z.z, u + 2, v, cam), p3 = point_of(z.w, u + 3, v, cam);
            float4* o = reinterpret_cast<float4*>(xyz) + 3 * g;
            o[0] = make_float4(p0.x, p0.y, p0.z, p1.x);
            o[1] = make_float4(p1.y, p1.z, p2.x, p2.y);
            o[2] = make_float4(p2.z, p3.x, p3.y, p3.z);
        } else {
            for (size_t i = i0; i < i0 + 4 && i < n; i++) {
                const int v = (int)(i / (size_t)W), u = (int)(i - (size_t)v * W);
                const float3 p = point_of(depth[i], u, v, cam);
                xyz[3 * i] = p.x;
                xyz[3 * i + 1] = p.y;
                xyz[3 * i + 2] = p.z;
            }
        }
    }
}

// One CTA per 32 x TH output tile; Z and validity planes of the tile plus a
// halo of rn staged in shared memory (validity as the full path stages it:
// 1 valid, +inf not).
template <int TH>
__global__ void __launch_bounds__(TILE_W * TH)
    k_initial_normals(const float* __restrict__ depth, int H, int W, Camera cam, int rn, float det_tol,
                      float* __restrict__ normal) {
    extern __shared__ float smem[];
    constexpr int NT = TILE_W * TH;
    const int SW = TILE_W + 2 * rn, SH = TH + 2 * rn;
    float* tz = smem;
    float* tcv = smem + SW * SH;
    const int ub = blockIdx.x * TILE_W, vb = blockIdx.y * TH;
    const int tid = threadIdx.y * TILE_W + threadIdx.x;
    for (int i = tid; i < SW * SH; i += NT) {
        const int sy = i / SW, sx = i - sy * SW;
        const int gv = vb - rn + sy, gu = ub - rn + sx;
        float z = 0.f, c = __int_as_float(0x7f800000);
        if (gu >= 0 && gu < W && gv >= 0 && gv < H) {
            const float d = __ldg(depth + (size_t)gv * W + gu);
            if (range_ok(d)) {
                z = d;
                c = 1.f;
            }
        }
        tz[i] = z;
        tcv[i] = c;
    }
    __syncthreads();
    const int u0 = ub + threadIdx.x, v0 = vb + threadIdx.y;
    if (u0 >= W || v0 >= H) return;
    const int cidx = (threadIdx.y + rn) * SW + threadIdx.x + rn;
    const float Zp = tz[cidx];
    float nx = 0.f, ny = 0.f, nz = 1.f;
    bool ok = tcv[cidx] == 1.f;
    if (ok)
        ok = initial_normal(tz + cidx, tcv + cidx, SW, rn, (float)u0 - cam.cx, (float)v0 - cam.cy, Zp, cam,
                            det_tol, nx, ny, nz);
    const size_t out = (size_t)v0 * W + u0;
    const float q = __int_as_float(0x7fffffff);
    normal[3 * out] = ok ? nx : q;
    normal[3 * out + 1] = ok ? ny : q;
    normal[3 * out + 2] = ok ? nz : q;
}

constexpr int NORMAL_TH = 8;

}  // namespace

cudaError_t launch_backproject(const float* depth, int H, int W, const Camera& cam, float* xyz, int sms,
                               cudaStream_t stream) {
    const size_t groups = ((size_t)H * W + 3) / 4;
    const size_t want = (groups + BP_THREADS - 1) / BP_THREADS;
    const size_t cap = (size_t)(sms > 0 ? sms : 152) * 8;  // 8 resident CTAs of 256 threads per SM
    const int grid = (int)(want < cap ? want : cap);
    const bool vec = ((uintptr_t)depth & 15u) == 0 && ((uintptr_t)xyz & 15u) == 0 && (W & 3) == 0;
    if (vec)
        k_backproject<true><<<grid, BP_THREADS, 0, stream>>>(depth, H, W, cam, xyz);
    else
        k_backproject<false><<<grid, BP_THREADS, 0, stream>>>(depth, H, W, cam, xyz);
    return cudaGetLastError();
}

size_t initial_normals_smem_bytes(int rn) {
    return (size_t)(TILE_W + 2 * rn) * (NORMAL_TH + 2 * rn) * 2 * sizeof(float);
}

cudaError_t launch_initial_normals(const float* depth, int H, int W, const Camera& cam, int rn, float det_tol,
                                   float* normal, cudaStream_t stream) {
    const dim3 block(TILE_W, NORMAL_TH);
    const dim3 grid((W + TILE_W - 1) / TILE_W, (H + NORMAL_TH - 1) / NORMAL_TH);
    k_initial_normals<NORMAL_TH><<<grid, block, initial_normals_smem_bytes(rn), stream>>>(depth, H, W, cam, rn,
                                                                                       det_tol, normal);
    return cudaGetLastError();
}

}  // namespace pcurv
