// pc_f32x2.cuh -- packed single-precision pairs for sm_100-family GPUs.
//
// Blackwell executes add/mul/fma on two FP32 values held in a 64-bit register
// pair as one instruction (PTX add/mul/fma .rn.f32x2).  Each half is rounded
// exactly like the scalar instruction, so a pair computes two independent
// IEEE results while taking one issue slot.
#pragma once
#include <cuda_runtime.h>

namespace pcurv {

typedef unsigned long long f32x2;  // (lo, hi) single-precision pair

__device__ __forceinline__ f32x2 pack(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 splat(float x) { return pack(x, x); }

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// sum of the two halves
__device__ __forceinline__ float hsum(f32x2 v) {
    float a, b;
    unpack(v, a, b);
    return a + b;
}

}  // namespace pcurv
