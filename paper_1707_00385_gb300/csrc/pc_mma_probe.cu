// pc_mma_probe.cu -- pc_moments_probe: a design measurement, not part of the
// method.  It times the step that dominates the curvature kernels -- the
// window moments of one re-weighted iteration (Sec. 3.2.3, Eq.
// iter_reweighted_update: the 21 entries of J^T W J and the 6 of J^T W eps,
// summed over every window point) -- in two forms on the same synthetic
// windows, so that the tensor-core recast of the moments can be judged by
// measurement:
//
//   mode 0  packed FP32 multiply-adds into registers, as the curvature
//           kernels accumulate them (20 sums of J^T W J, 6 of J^T W eps);
//   mode 1  tensor cores: each point's features f = sqrt(w) (-j0, j1, 1, x^2,
//           x y, y^2) are split into TF32 hi + lo parts, staged in shared
//           memory per warp, and J^T W J = sum f f^T is accumulated by
//           mma.sync m16n8k8 TF32 with three products per block (hi hi,
//           hi lo, lo hi: single-precision accuracy; one TF32 product alone
//           moves most pixels beyond the parity tolerance).  The Gram of one
//           pixel has no operand in common with another pixel's, so one MMA
//           serves two pixels through a block-diagonal K: rows 0-5 are pixel
//           P's features over K = its 4 points, rows 8-13 pixel Q's over the
//           other 4 (each lane then holds the same two values as its A and B
//           fragments).  J^T W eps stays on the FP32 pipe.
//
// Both modes share the per-point front end of the curvature kernels (local
// coordinates from a staged range tile, residual, Cauchy weight, Jacobian
// rows, in packed pairs) and run T iterations over a 15 x 15 window per
// pixel; each thread folds its sums into one float so no work is removed.
#include <cuda_runtime.h>

#include "../../include/pcurv.h"
#include "pc_f32x2.cuh"

namespace {

using namespace pcurv;

constexpr int R = 7;                    // window radius: 15 x 15 points
constexpr int TW = 32, TH = 8;          // one thread per pixel of a 32 x 8 tile
constexpr int SW = TW + 2 * R, SH = TH + 2 * R;
constexpr int NT = TW * TH;
constexpr int PTS = 4;                  // points per thread per MMA step (two symmetric pairs)
constexpr int FSTRIDE = PTS * 8 * 2;    // staged floats per lane: 4 points x 8 features x (hi, lo)
constexpr int TILE_FLOATS = (SW * SH + 63) / 64 * 64;
static_assert(FSTRIDE == 64, "a warp's Grams (32 pixels x 64 floats) reuse its feature region");

size_t probe_smem_bytes(int mode) { return (TILE_FLOATS + (mode == 1 ? NT * FSTRIDE : 0)) * sizeof(float); }

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ unsigned tf32_of(float x) {
    unsigned y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

// d += A B for one m16n8k8 TF32 block: a = {a0, 0, 0, a3}, b = {b0, b1}
__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(0u), "r"(0u), "r"(a3), "r"(b0), "r"(b1));
}

// Per-iteration constants of one pixel (splat into pairs), as in the curvature kernels.
struct Coef {
    f32x2 cx0, cx1, cx2, bx, by, bh, ga, gb, gc, nhs, nts, nzp;
};

// x, y, hs of a symmetric pair, its scaled residual e and Jacobian rows.
__device__ __forceinline__ void front(const Coef& k, f32x2 Z, f32x2 DU, f32x2 RX, f32x2 RY, f32x2 RH, f32x2& X,
                                      f32x2& Y, f32x2& E, f32x2& NJ0, f32x2& J1) {
    const f32x2 dZ = add2(Z, k.nzp);
    X = fma2(fma2(DU, k.cx0, RX), Z, mul2(k.bx, dZ));
    Y = fma2(fma2(DU, k.cx1, RY), Z, mul2(k.by, dZ));
    const f32x2 Hs = fma2(fma2(DU, k.cx2, RH), Z, mul2(k.bh, dZ));
    const f32x2 GA = fma2(k.ga, X, mul2(k.gb, Y));
    const f32x2 GB = fma2(k.gb, X, mul2(k.gc, Y));
    E = fma2(GA, X, fma2(GB, Y, fma2(k.nhs, Hs, k.nts)));
    NJ0 = fma2(GB, Hs, Y);
    J1 = fma2(GA, Hs, X);
}

template <int MODE>
__global__ void __launch_bounds__(NT, MODE == 0 ? 2 : 1)
    k_moments(int tasks, int iters, float* __restrict__ sink) {
    // dynamic: the range tile, then (mode 1) the staged features of every
    // lane, whose region each warp reuses for its pixels' Grams at the end
    extern __shared__ float dsm[];
    float* tz = dsm;
    float* feat = dsm + TILE_FLOATS;
    const int tid = threadIdx.y * TW + threadIdx.x;
    const int lane = threadIdx.x, warp = threadIdx.y;
    float check = 0.f;
    for (int task = blockIdx.x; task < tasks; task += gridDim.x) {
        // a smooth synthetic range tile (0.9 - 1.5 m) with a per-task tilt
        __syncthreads();
        for (int i = tid; i < SW * SH; i += NT) {
            const float u = (float)(i % SW), v = (float)(i / SW);
            tz[i] = 1.2f + 0.002f * u - 0.0015f * v + 0.3f * __sinf(0.05f * (u + task) + 0.07f * v);
        }
        __syncthreads();
        const float* zc = tz + (threadIdx.y + R) * SW + threadIdx.x + R;
        const float Zp = *zc;
        float Rm[9] = {0.99f, -0.01f, -0.1f, 0.0f, 0.995f, -0.1f, 0.1f, 0.1f, 0.99f};
        float A = 0.5f, B = 0.1f, C = -0.3f, t = 0.001f;
        for (int it = 0; it < iters; it++) {
            Coef k;
            const float ifx = 1.f / 525.f, sig = 100.f, hs = 2.f / sig;
            const float ap = (float)(threadIdx.x) - 16.f, bp = (float)(threadIdx.y) - 4.f;
            const float cx0 = Rm[0] * ifx, cy0 = Rm[1] * ifx, cx1 = Rm[3] * ifx, cy1 = Rm[4] * ifx;
            const float cx2 = Rm[6] * ifx, cy2 = Rm[7] * ifx;
            k.cx0 = splat(cx0); k.cx1 = splat(cx1); k.cx2 = splat(cx2 * hs);
            k.bx = splat(fmaf(cx0, ap, fmaf(cy0, bp, Rm[2])));
            k.by = splat(fmaf(cx1, ap, fmaf(cy1, bp, Rm[5])));
            k.bh = splat(fmaf(cx2, ap, fmaf(cy2, bp, Rm[8])) * hs);
            k.ga = splat(0.5f * sig * A); k.gb = splat(0.5f * sig * B); k.gc = splat(0.5f * sig * C);
            k.nhs = splat(-0.5f * sig * sig); k.nts = splat(-sig * t); k.nzp = splat(-Zp);
            const f32x2 CY0 = splat(cy0), CY1 = splat(cy1), CY2 = splat(cy2 * hs);
            // J^T W eps on the FP32 pipe in both modes
            f32x2 g0 = 0ull, g1 = 0ull, ge = 0ull, g3 = 0ull, g4 = 0ull, g5 = 0ull;
            float out = 0.f;
            if (MODE == 0) {
                f32x2 h00 = 0ull, h01 = 0ull, h11 = 0ull, s0 = 0ull, s1 = 0ull, h03 = 0ull, h04 = 0ull, h05 = 0ull,
                      h13 = 0ull, h14 = 0ull, h15 = 0ull, sw = 0ull, sxx = 0ull, sxy = 0ull, syy = 0ull,
                      m40 = 0ull, m31 = 0ull, m22 = 0ull, m13 = 0ull, m04 = 0ull;
                for (int dv = -R; dv <= 0; dv++) {
                    const float *za = zc + dv * SW, *zb = zc - dv * SW;
                    const f32x2 DV = pack((float)dv, -(float)dv);
                    f32x2 DU = pack(-(float)R, (float)R);
#pragma unroll
                    for (int du = -R; du <= R; du++) {
                        if (dv == 0 && du >= 0) break;
                        f32x2 X, Y, E, NJ0, J1;
                        front(k, pack(za[du], zb[-du]), DU, mul2(DV, CY0), mul2(DV, CY1), mul2(DV, CY2), X, Y,
                              E, NJ0, J1);
                        float ea, eb;
                        unpack(fma2(E, E, splat(1.f)), ea, eb);
                        const f32x2 Wt = pack(rcp_approx(ea), rcp_approx(eb));
                        const f32x2 XX = mul2(X, X), XY = mul2(X, Y), YY = mul2(Y, Y);
                        const f32x2 WE = mul2(Wt, E), WJ0 = mul2(Wt, NJ0), WJ1 = mul2(Wt, J1);
                        const f32x2 WXX = mul2(Wt, XX), WYY = mul2(Wt, YY);
                        s0 = add2(s0, WJ0); s1 = add2(s1, WJ1); sw = add2(sw, Wt);
                        sxx = add2(sxx, WXX); syy = add2(syy, WYY); ge = add2(ge, WE);
                        h00 = fma2(WJ0, NJ0, h00); h01 = fma2(WJ0, J1, h01);
                        h03 = fma2(WJ0, XX, h03); h04 = fma2(WJ0, XY, h04); h05 = fma2(WJ0, YY, h05);
                        h15 = fma2(WJ1, YY, h15); h14 = fma2(WJ1, XY, h14); h13 = fma2(WJ1, XX, h13);
                        h11 = fma2(WJ1, J1, h11);
                        g1 = fma2(WE, J1, g1); g0 = fma2(WE, NJ0, g0); g3 = fma2(WE, XX, g3);
                        g4 = fma2(WE, XY, g4); g5 = fma2(WE, YY, g5);
                        m04 = fma2(WYY, YY, m04); m13 = fma2(WYY, XY, m13); sxy = fma2(Wt, XY, sxy);
                        m31 = fma2(WXX, XY, m31); m40 = fma2(WXX, XX, m40); m22 = fma2(WXX, YY, m22);
                        DU = add2(DU, pack(1.f, -1.f));
                    }
                }
                out = hsum(h00) + hsum(h01) + hsum(h11) + hsum(s0) + hsum(s1) + hsum(h03) + hsum(h04) +
                      hsum(h05) + hsum(h13) + hsum(h14) + hsum(h15) + hsum(sw) + hsum(sxx) + hsum(sxy) +
                      hsum(syy) + hsum(m40) + hsum(m31) + hsum(m22) + hsum(m13) + hsum(m04);
            } else {
                float acc[16][4];
#pragma unroll
                for (int j = 0; j < 16; j++) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
                float* mine = feat + (warp * 32 + lane) * FSTRIDE;
                const float* wbase = feat + warp * 32 * FSTRIDE;
                const int g = lane >> 2, kk = lane & 3;
                int slot = 0;  // points staged so far in this step (0, 2)
                // 112 symmetric pairs + a padding pair: 56 full steps of 4 points, then one of 2 + 2 empty
                for (int dv = -R; dv <= 0; dv++) {
                    const float *za = zc + dv * SW, *zb = zc - dv * SW;
                    const f32x2 DV = pack((float)dv, -(float)dv);
                    f32x2 DU = pack(-(float)R, (float)R);
#pragma unroll
                    for (int du = -R; du <= R; du++) {
                        if (dv == 0 && du >= 0) break;
                        f32x2 X, Y, E, NJ0, J1;
                        front(k, pack(za[du], zb[-du]), DU, mul2(DV, CY0), mul2(DV, CY1), mul2(DV, CY2), X, Y,
                              E, NJ0, J1);
                        float ea, eb;
                        unpack(fma2(E, E, splat(1.f)), ea, eb);
                        const f32x2 S = pack(rsqrt_approx(ea), rsqrt_approx(eb));   // sqrt(w)
                        const f32x2 Wt = mul2(S, S);
                        const f32x2 XX = mul2(X, X), XY = mul2(X, Y), YY = mul2(Y, Y);
                        const f32x2 WE = mul2(Wt, E);
                        ge = add2(ge, WE);
                        g1 = fma2(WE, J1, g1); g0 = fma2(WE, NJ0, g0); g3 = fma2(WE, XX, g3);
                        g4 = fma2(WE, XY, g4); g5 = fma2(WE, YY, g5);
                        const f32x2 F[6] = {mul2(S, NJ0), mul2(S, J1), S, mul2(S, XX), mul2(S, XY), mul2(S, YY)};
#pragma unroll
                        for (int f = 0; f < 6; f++) {
                            float fa, fb;
                            unpack(F[f], fa, fb);
                            const float ha = __uint_as_float(tf32_of(fa)), hb = __uint_as_float(tf32_of(fb));
                            reinterpret_cast<float2*>(mine)[(slot * 8 + f)] = make_float2(ha, fa - ha);
                            reinterpret_cast<float2*>(mine)[((slot + 1) * 8 + f)] = make_float2(hb, fb - hb);
                        }
                        reinterpret_cast<float4*>(mine)[(slot * 8 + 6) / 2] = make_float4(0.f, 0.f, 0.f, 0.f);
                        reinterpret_cast<float4*>(mine)[((slot + 1) * 8 + 6) / 2] = make_float4(0.f, 0.f, 0.f, 0.f);
                        slot += 2;
                        const bool last = dv == 0 && du == -1;
                        if (slot == PTS || last) {
                            if (slot < PTS) {  // a short last step: the missing points weigh nothing
                                for (int f = slot * 16; f < PTS * 16; f++) mine[f] = 0.f;
                            }
                            __syncwarp();
#pragma unroll
                            for (int j = 0; j < 16; j++) {
                                const float2 P = reinterpret_cast<const float2*>(wbase + (2 * j) * FSTRIDE)[kk * 8 + g];
                                const float2 Q =
                                    reinterpret_cast<const float2*>(wbase + (2 * j + 1) * FSTRIDE)[kk * 8 + g];
                                const unsigned ph = __float_as_uint(P.x), qh = __float_as_uint(Q.x);
                                const unsigned pl = tf32_of(P.y), ql = tf32_of(Q.y);
                                mma_tf32(acc[j], ph, qh, ph, qh);
                                mma_tf32(acc[j], ph, qh, pl, ql);
                                mma_tf32(acc[j], pl, ql, ph, qh);
                            }
                            __syncwarp();
                            slot = 0;
                        }
                        DU = add2(DU, pack(1.f, -1.f));
                    }
                }
                // each pixel's Gram to its own lane through shared memory
                float* gw = feat + warp * 32 * FSTRIDE;
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    gw[(2 * j) * 64 + g * 8 + 2 * kk] = acc[j][0];
                    gw[(2 * j) * 64 + g * 8 + 2 * kk + 1] = acc[j][1];
                    gw[(2 * j + 1) * 64 + g * 8 + 2 * kk] = acc[j][2];
                    gw[(2 * j + 1) * 64 + g * 8 + 2 * kk + 1] = acc[j][3];
                }
                __syncwarp();
#pragma unroll
                for (int a = 0; a < 6; a++)
#pragma unroll
                    for (int b = a; b < 6; b++) out += gw[lane * 64 + a * 8 + b];
                __syncwarp();
            }
            out += hsum(g0) + hsum(g1) + hsum(ge) + hsum(g3) + hsum(g4) + hsum(g5);
            check += out;
            // a small change of the state, as a solve would make
            A += 1e-3f * out;
            t -= 1e-9f * out;
            Rm[2] += 1e-9f * out;
        }
    }
    sink[blockIdx.x * NT + tid] = check;
}

}  // namespace

extern "C" pc_status pc_moments_probe(int mode, int pixels, int iters, float* sink, long long sink_len,
                                      void* stream, int* blocks_out) {
    if ((mode != 0 && mode != 1) || pixels <= 0 || iters <= 0 || !sink || ((size_t)sink & 3u))
        return PC_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PC_ERR_CUDA;
    const int tasks = (pixels + NT - 1) / NT;
    int per_sm = 0;
    const size_t smem = probe_smem_bytes(mode);
    cudaError_t e;
    if (mode == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_moments<0>, NT, smem);
    } else {
        e = cudaFuncSetAttribute(k_moments<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_moments<1>, NT, smem);
    }
    if (e != cudaSuccess) return PC_ERR_CUDA;
    int blocks = sms * (per_sm > 0 ? per_sm : 1);
    if (blocks > tasks) blocks = tasks;
    if (sink_len < (long long)blocks * NT) return PC_ERR_INVALID_ARG;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, sink) != cudaSuccess) {
        cudaGetLastError();
        return PC_ERR_INVALID_ARG;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PC_ERR_INVALID_ARG;
    const dim3 block(TW, TH);
    if (mode == 0)
        k_moments<0><<<blocks, block, smem, (cudaStream_t)stream>>>(tasks, iters, sink);
    else
        k_moments<1><<<blocks, block, smem, (cudaStream_t)stream>>>(tasks, iters, sink);
    if (cudaGetLastError() != cudaSuccess) return PC_ERR_CUDA;
    if (blocks_out) *blocks_out = blocks;
    return PC_OK;
}
