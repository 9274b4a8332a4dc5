// pc_pack.cu -- float32 ranges to per-tile-centred 16-bit storage.
//
// One CTA per 32x8 tile: the tile's base is the midpoint of its smallest and
// largest valid range (so the offsets are as small as the tile allows), and
// each pixel stores range - base rounded to the nearest FP16 or BF16 value;
// pixels without a valid range store NaN.
#include <cfloat>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pc_internal.h"

namespace pcurv {

constexpr int PACK_THREADS = TILE_W * PACK_TILE_H;

__global__ void __launch_bounds__(PACK_THREADS)
    k_pack(const float* __restrict__ depth, int H, int W, int format, unsigned short* __restrict__ packed,
           float* __restrict__ tile_base) {
    __shared__ float s_lo[PACK_THREADS / 32], s_hi[PACK_THREADS / 32];
    const int u = blockIdx.x * TILE_W + threadIdx.x, v = blockIdx.y * PACK_TILE_H + threadIdx.y;
    const int tid = threadIdx.y * TILE_W + threadIdx.x;
    const bool inside = u < W && v < H;
    const float d = inside ? depth[(size_t)v * W + u] : 0.f;
    const bool valid = inside && d > 0.f && d <= FLT_MAX;
    float lo = valid ? d : FLT_MAX, hi = valid ? d : -FLT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((tid & 31) == 0) {
        s_lo[tid >> 5] = lo;
        s_hi[tid >> 5] = hi;
    }
    __syncthreads();
    lo = s_lo[0];
    hi = s_hi[0];
#pragma unroll
    for (int i = 1; i < PACK_THREADS / 32; i++) {
        lo = fminf(lo, s_lo[i]);
        hi = fmaxf(hi, s_hi[i]);
    }
    const float base = lo <= hi ? 0.5f * (lo + hi) : 0.f;
    if (tid == 0) tile_base[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = base;
    if (!inside) return;
    const float off = valid ? d - base : __int_as_float(0x7fffffff);
    packed[(size_t)v * W + u] = format == 1 ? __half_as_ushort(__float2half_rn(off))
                                            : __bfloat16_as_ushort(__float2bfloat16_rn(off));
}

cudaError_t launch_pack(const float* depth, int H, int W, int format, unsigned short* packed,
                        float* tile_base, cudaStream_t stream) {
    const dim3 block(TILE_W, PACK_TILE_H);
    const dim3 grid((W + TILE_W - 1) / TILE_W, (H + PACK_TILE_H - 1) / PACK_TILE_H);
    k_pack<<<grid, block, 0, stream>>>(depth, H, W, format, packed, tile_base);
    return cudaGetLastError();
}

}  // namespace pcurv
