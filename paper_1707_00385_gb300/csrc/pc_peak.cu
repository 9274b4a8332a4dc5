// pc_peak.cu -- pc_fp32_peak_kernel: a measurement utility, not part of the
// method.  It measures the single-precision issue ceiling that the curvature
// kernels are judged against: every thread runs independent chains of fused
// multiply-adds (packed FP32x2 pairs or scalar), long enough that launch and
// tail costs vanish, so a timed launch gives the FP32 FLOP/s the GPU sustains
// at its current clock.
#include <cuda_runtime.h>

#include "../../include/pcurv.h"
#include "pc_f32x2.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 16;  // independent accumulators per thread

// a_i <- a_i * b + c for every chain, iters rounds.  b and c are the same
// registers in every instruction (operand reuse, the pipe's best case); b is
// a hair below 1 and c tiny, so the values stay finite for any round count.
__global__ void __launch_bounds__(kThreads) k_fma2(int iters, float b0, float c0, float* sink) {
    using namespace pcurv;
    const f32x2 b = splat(b0), c = splat(c0);
    f32x2 a[kChains];
#pragma unroll
    for (int i = 0; i < kChains; i++) a[i] = pack((float)threadIdx.x + i, (float)blockIdx.x - i);
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < kChains; i++) a[i] = fma2(a[i], b, c);
    }
    f32x2 s = a[0];
#pragma unroll
    for (int i = 1; i < kChains; i++) s = add2(s, a[i]);
    sink[blockIdx.x * kThreads + threadIdx.x] = hsum(s);
}

__global__ void __launch_bounds__(kThreads) k_fma1(int iters, float b, float c, float* sink) {
    float a[2 * kChains];
#pragma unroll
    for (int i = 0; i < 2 * kChains; i++) a[i] = (float)threadIdx.x + i;
    for (int k = 0; k < iters; k++) {
#pragma unroll
        for (int i = 0; i < 2 * kChains; i++) a[i] = __fmaf_rn(a[i], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kChains; i++) s += a[i];
    sink[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" pc_status pc_fp32_peak_kernel(int blocks, int iters, int packed, float* sink, long long sink_len,
                                         void* stream, double* flop_out) {
    if (blocks <= 0 || iters <= 0 || !sink || ((unsigned long long)(size_t)sink & 3u) ||
        sink_len < (long long)blocks * kThreads)
        return PC_ERR_INVALID_ARG;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, sink) != cudaSuccess) {
        cudaGetLastError();
        return PC_ERR_INVALID_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (packed)
        k_fma2<<<blocks, kThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
    else
        k_fma1<<<blocks, kThreads, 0, s>>>(iters, 0.9999999f, 1e-7f, sink);
    if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
    // two FLOP per fused multiply-add, 2 kChains multiply-adds per thread and round
    if (flop_out) *flop_out = 2.0 * 2.0 * kChains * (double)iters * kThreads * blocks;
    return PC_OK;
}
