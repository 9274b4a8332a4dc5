// pc_fit.cuh -- the fused per-pixel curvature kernel (sm_103a).
//
// One CTA computes a 32 x 8 tile of output pixels, one thread per pixel.  The
// CTA first stages the tile's range values plus a halo of max(r, r_n) pixels
// into shared memory as (Z, c) pairs, c = 1 for a valid range and +inf for
// none (outside the image, zero, negative or not finite).  Each thread then
// runs the whole method of Spek, Li and Drummond (arXiv 1707.00385, Sec. 3.2)
// for its pixel in registers:
//
//   initial normal   Sec. 3.2.1, Eq. initialnormal (7x7 regression)
//   frame            Sec. 3.2.2 (minimal rotation to the normal, A=B=C=t_z=0)
//   T iterations     Sec. 3.2.3: residuals of Eq. quad, Jacobian, weights of
//                    Eq. weighting_function, the 6x6 system of
//                    Eq. iter_reweighted_update solved by a Jacobi-scaled
//                    LDL^T factorisation, Gauss-Newton update
//   eigen step       Sec. 3.1.2 (T1, T2 closed form), refined normal Sec. 3.2.4
//
// The hot loop visits every window point once per iteration.  Its arithmetic
// is arranged for FP32 issue rate and for accuracy:
//   * p'_i = p_i - p is never formed from absolute coordinates.  With
//     dZ = Z_i - Z_p (exact for ranges within a factor 2),
//       X_i - X_p = ((u_i - u_p) Z_i + (u_p - c_x) dZ) / f_x,
//     and the local coordinate x = R_0 . p'_i becomes
//       x = Z_i * alpha_x(du, dv) + dZ * beta_x,
//     alpha_x = du R00/f_x + dv R01/f_y, beta_x = R00 (u_p-c_x)/f_x +
//     R01 (v_p-c_y)/f_y + R02, both per iteration; likewise y and h.
//   * the weight k/(k + eps^2) is 1/(1 + eps^2/k + [invalid]*inf), one fused
//     multiply-add and one hardware reciprocal; invalid points get weight
//     exactly 0 without a branch.
//   * J^T W J needs 21 entries and J^T W eps 6; they come from 26 running
//     sums, because with j = (j0, j1, -1, x^2/2, x y, y^2/2) the (A,B,C)
//     block only has five distinct moments (H_AC and H_BB share x^2 y^2) and
//     the t_z row is sums of w j.
#pragma once
#include <cfloat>
#include <cuda_runtime.h>

#include "pc_internal.h"

namespace pcurv {

__device__ __forceinline__ float rcp_approx(float x) {
    // PTX rcp.approx.ftz.f32: at most 1 ulp of error; rcp(+inf) = +0.
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fffffff); }

// 26 running sums of one iteration (see the header comment).
struct Moments {
    float h00, h01, h11;       // sum w j0 j0, w j0 j1, w j1 j1
    float s0, s1;              // sum w j0, w j1           (t_z column, times -1)
    float h03, h04, h05;       // sum w j0 x^2, w j0 x y, w j0 y^2
    float h13, h14, h15;       // sum w j1 x^2, w j1 x y, w j1 y^2
    float sw;                  // sum w                    (t_z, t_z)
    float sxx, sxy, syy;       // sum w x^2, w x y, w y^2  (t_z row, times -1)
    float m40, m31, m22, m13, m04;  // sum w x^4, w x^3 y, w x^2 y^2, w x y^3, w y^4
    float g0, g1, ge, g3, g4, g5;   // sum w eps j0, w eps j1, w eps, w eps x^2, w eps x y, w eps y^2
};

// Per-iteration constants of one pixel.
struct Coef {
    float cx0, cy0, bx;   // x = Z (du cx0 + dv cy0) + dZ bx
    float cx1, cy1, by;   // y
    float cx2, cy2, bh;   // h (local z before the offset t_z)
    float hA, hC;         // A/2, C/2
    float A, B, C, tz;
    float invk, Zp;
};

__device__ __forceinline__ void zero(Moments& m) {
    m.h00 = m.h01 = m.h11 = m.s0 = m.s1 = 0.f;
    m.h03 = m.h04 = m.h05 = m.h13 = m.h14 = m.h15 = 0.f;
    m.sw = m.sxx = m.sxy = m.syy = 0.f;
    m.m40 = m.m31 = m.m22 = m.m13 = m.m04 = 0.f;
    m.g0 = m.g1 = m.ge = m.g3 = m.g4 = m.g5 = 0.f;
}

// Local coordinates (x, y, h) of one window point.
__device__ __forceinline__ void local_xyz(const Coef& k, float Z, float du, float rx, float ry,
                                          float rh, float& x, float& y, float& h) {
    const float dZ = Z - k.Zp;
    x = fmaf(fmaf(du, k.cx0, rx), Z, k.bx * dZ);
    y = fmaf(fmaf(du, k.cx1, ry), Z, k.by * dZ);
    h = fmaf(fmaf(du, k.cx2, rh), Z, k.bh * dZ);
}

// One point visit: residual (Eq. quad in the local frame), weight, Jacobian,
// and the 26 sums.  c = 1 for a valid point, +inf for none.
template <bool REJECT>
__device__ __forceinline__ void visit(Moments& m, const Coef& k, float Z, float c, float du,
                                      float rx, float ry, float rh, float thr) {
    float x, y, h;
    local_xyz(k, Z, du, rx, ry, rh, x, y, h);
    const float xx = x * x, xy = x * y, yy = y * y;
    // eps = A/2 x^2 + B x y + C/2 y^2 - (h + t_z)
    const float eps = fmaf(k.hA, xx, fmaf(k.B, xy, fmaf(k.hC, yy, -(h + k.tz))));
    const float e2 = eps * eps;
    float w = rcp_approx(fmaf(e2, k.invk, c));
    if (REJECT) w = (e2 <= thr) ? w : 0.f;
    // d eps / d theta_x = -(B x + C y) h - y ; d eps / d theta_y = (A x + B y) h + x
    const float j0 = fmaf(-fmaf(k.B, x, k.C * y), h, -y);
    const float j1 = fmaf(fmaf(k.A, x, k.B * y), h, x);
    const float we = w * eps;
    const float wj0 = w * j0, wj1 = w * j1;
    const float wxx = w * xx, wxy = w * xy, wyy = w * yy;
    m.h00 = fmaf(wj0, j0, m.h00);
    m.h01 = fmaf(wj0, j1, m.h01);
    m.h11 = fmaf(wj1, j1, m.h11);
    m.s0 += wj0;
    m.s1 += wj1;
    m.h03 = fmaf(wj0, xx, m.h03);
    m.h04 = fmaf(wj0, xy, m.h04);
    m.h05 = fmaf(wj0, yy, m.h05);
    m.h13 = fmaf(wj1, xx, m.h13);
    m.h14 = fmaf(wj1, xy, m.h14);
    m.h15 = fmaf(wj1, yy, m.h15);
    m.sw += w;
    m.sxx += wxx;
    m.sxy += wxy;
    m.syy += wyy;
    m.m40 = fmaf(wxx, xx, m.m40);
    m.m31 = fmaf(wxx, xy, m.m31);
    m.m22 = fmaf(wxx, yy, m.m22);
    m.m13 = fmaf(wxy, yy, m.m13);
    m.m04 = fmaf(wyy, yy, m.m04);
    m.g0 = fmaf(we, j0, m.g0);
    m.g1 = fmaf(we, j1, m.g1);
    m.ge += we;
    m.g3 = fmaf(we, xx, m.g3);
    m.g4 = fmaf(we, xy, m.g4);
    m.g5 = fmaf(we, yy, m.g5);
}

// Squared residual of a valid point, 0 for an invalid one (rejection pre-pass).
__device__ __forceinline__ float sq_residual(const Coef& k, float Z, float c, float du, float rx,
                                             float ry, float rh) {
    float x, y, h;
    local_xyz(k, Z, du, rx, ry, rh, x, y, h);
    const float eps = fmaf(k.hA, x * x, fmaf(k.B, x * y, fmaf(k.hC, y * y, -(h + k.tz))));
    return c == 1.f ? eps * eps : 0.f;
}

// Solves (J^T W J) b = J^T W eps from the 26 sums, b returned as the update
// delta = -b.  Jacobi-scaled LDL^T: S = D H D, D = diag(H)^-1/2; singular when
// a diagonal entry is <= 0 or a pivot of S is <= pivot_tol.
__device__ __forceinline__ bool solve_update(const Moments& m, float pivot_tol, float delta[6]) {
    float H[6][6];
    H[0][0] = m.h00; H[0][1] = m.h01; H[0][2] = -m.s0;
    H[0][3] = 0.5f * m.h03; H[0][4] = m.h04; H[0][5] = 0.5f * m.h05;
    H[1][1] = m.h11; H[1][2] = -m.s1;
    H[1][3] = 0.5f * m.h13; H[1][4] = m.h14; H[1][5] = 0.5f * m.h15;
    H[2][2] = m.sw; H[2][3] = -0.5f * m.sxx; H[2][4] = -m.sxy; H[2][5] = -0.5f * m.syy;
    H[3][3] = 0.25f * m.m40; H[3][4] = 0.5f * m.m31; H[3][5] = 0.25f * m.m22;
    H[4][4] = m.m22; H[4][5] = 0.5f * m.m13;
    H[5][5] = 0.25f * m.m04;
    const float g[6] = {m.g0, m.g1, -m.ge, 0.5f * m.g3, m.g4, 0.5f * m.g5};
    float D[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        if (!(H[i][i] > 0.f)) return false;
        D[i] = rsqrtf(H[i][i]);
    }
    float S[6][6], L[6][6], d[6];
#pragma unroll
    for (int i = 0; i < 6; i++)
#pragma unroll
        for (int j = i; j < 6; j++) S[i][j] = H[i][j] * D[i] * D[j];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        float dj = S[j][j];
#pragma unroll
        for (int k = 0; k < j; k++) dj -= L[j][k] * L[j][k] * d[k];
        if (!(dj > pivot_tol)) return false;
        d[j] = dj;
        const float idj = 1.f / dj;
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            float s = S[j][i];
#pragma unroll
            for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k] * d[k];
            L[i][j] = s * idj;
        }
    }
    float z[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float s = D[i] * g[i];
#pragma unroll
        for (int k = 0; k < i; k++) s -= L[i][k] * z[k];
        z[i] = s;
    }
#pragma unroll
    for (int i = 0; i < 6; i++) z[i] /= d[i];
#pragma unroll
    for (int i = 5; i >= 0; i--) {
        float s = z[i];
#pragma unroll
        for (int k = i + 1; k < 6; k++) s -= L[k][i] * z[k];
        z[i] = s;
    }
#pragma unroll
    for (int i = 0; i < 6; i++) delta[i] = -D[i] * z[i];
    return true;
}

// R <- Rot(t0, t1, 0) R, Rot the rotation by angle |t| about t/|t|
// (Rodrigues: I + sin(th)/th [t]x + (1 - cos th)/th^2 [t]x^2).
__device__ __forceinline__ void rotate_left(float R[9], float t0, float t1) {
    const float th2 = fmaf(t0, t0, t1 * t1);
    float sa = 1.f, c1 = 0.5f;
    if (th2 > 0.f) {
        const float th = sqrtf(th2);
        float s, c;
        sincosf(0.5f * th, &s, &c);
        sa = 2.f * s * c / th;
        c1 = 2.f * s * s / th2;
    }
    const float q[9] = {1.f - c1 * t1 * t1, c1 * t0 * t1,       sa * t1,
                        c1 * t0 * t1,       1.f - c1 * t0 * t0, -sa * t0,
                        -sa * t1,           sa * t0,            1.f - c1 * th2};
    float o[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            o[3 * i + j] = fmaf(q[3 * i], R[j], fmaf(q[3 * i + 1], R[3 + j], q[3 * i + 2] * R[6 + j]));
#pragma unroll
    for (int i = 0; i < 9; i++) R[i] = o[i];
}

// RW > 0: window radius fixed at compile time, dense window, columns unrolled.
// RW == 0: radius and stride from cfg.
template <int RW, bool REJECT>
__global__ void __launch_bounds__(BLOCK_THREADS)
    k_fit(const float* __restrict__ depth, int H, int W, Camera cam, FitConfig cfg,
          float* __restrict__ k1o, float* __restrict__ k2o, float* __restrict__ nrmo) {
    extern __shared__ float2 tile[];
    const int r = RW > 0 ? RW : cfg.r;
    const int s = RW > 0 ? 1 : cfg.stride;
    const int r0 = (r / s) * s;   // first sampled offset is -r0
    const int halo = r > cfg.rn ? r : cfg.rn;
    const int SW = TILE_W + 2 * halo;
    const int SH = TILE_H + 2 * halo;
    const int ub = blockIdx.x * TILE_W, vb = blockIdx.y * TILE_H;
    const int tid = threadIdx.y * TILE_W + threadIdx.x;

    // stage the tile + halo (Sec. 3.2, first item: the range image)
    for (int i = tid; i < SW * SH; i += BLOCK_THREADS) {
        const int sy = i / SW, sx = i - sy * SW;
        const int gv = vb - halo + sy, gu = ub - halo + sx;
        float z = 0.f, c = __int_as_float(0x7f800000);
        if (gu >= 0 && gu < W && gv >= 0 && gv < H) {
            const float d = __ldg(depth + (size_t)gv * W + gu);
            if (d > 0.f && d <= FLT_MAX) {
                z = d;
                c = 1.f;
            }
        }
        tile[i] = make_float2(z, c);
    }
    __syncthreads();

    const int u0 = ub + threadIdx.x, v0 = vb + threadIdx.y;
    if (u0 >= W || v0 >= H) return;
    const size_t out = (size_t)v0 * W + u0;
    const float2* ctr = tile + (threadIdx.y + halo) * SW + threadIdx.x + halo;
    const float Zp = ctr->x;
    const float ap = (float)u0 - cam.cx, bp = (float)v0 - cam.cy;
    bool ok = ctr->y == 1.f;

    // ---- initial normal: z = a x + b y + c over the valid (2rn+1)^2 patch
    float nx = 0.f, ny = 0.f, nz = 1.f;
    if (ok) {
        float n = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f, sxz = 0.f,
              syz = 0.f;
        for (int dv = -cfg.rn; dv <= cfg.rn; dv++) {
            const float2* row = ctr + dv * SW;
            for (int du = -cfg.rn; du <= cfg.rn; du++) {
                const float2 e = row[du];
                if (e.y == 1.f) {
                    const float dZ = e.x - Zp;
                    const float X = fmaf((float)du, e.x, ap * dZ) * cam.ifx;
                    const float Y = fmaf((float)dv, e.x, bp * dZ) * cam.ify;
                    n += 1.f;
                    sx += X; sy += Y; sz += dZ;
                    sxx = fmaf(X, X, sxx); sxy = fmaf(X, Y, sxy); syy = fmaf(Y, Y, syy);
                    sxz = fmaf(X, dZ, sxz); syz = fmaf(Y, dZ, syz);
                }
            }
        }
        // centred second moments M and v (shift by the centre point first)
        const float in = 1.f / n;
        const float mx = sx * in, my = sy * in, mz = sz * in;
        const float m00 = fmaf(-sx, mx, sxx), m01 = fmaf(-sx, my, sxy), m11 = fmaf(-sy, my, syy);
        const float w0 = fmaf(-sx, mz, sxz), w1 = fmaf(-sy, mz, syz);
        const float det = fmaf(m00, m11, -m01 * m01), tr = m00 + m11;
        if (n < 3.f || !(det > cfg.det_tol * tr * tr)) {
            ok = false;
        } else {
            const float a = (m11 * w0 - m01 * w1) / det;
            const float b = (m00 * w1 - m01 * w0) / det;
            const float sc = rsqrtf(fmaf(a, a, fmaf(b, b, 1.f)));
            nx = -a * sc; ny = -b * sc; nz = sc;
        }
    }

    // ---- window count
    if (ok) {
        int cnt = 0;
        for (int dv = -r0; dv <= r; dv += s) {
            const float2* row = ctr + dv * SW;
            if (RW > 0) {
#pragma unroll
                for (int du = -RW; du <= RW; du++) cnt += row[du].y == 1.f;
            } else {
                for (int du = -r0; du <= r; du += s) cnt += row[du].y == 1.f;
            }
        }
        ok = cnt >= cfg.min_window;
    }

    float R[9];
    float A = 0.f, B = 0.f, C = 0.f, tz = 0.f;
    {
        // minimal rotation with R n = e_z: I + [w]x + [w]x^2/(1+n_z), w = n x e_z
        const float f = 1.f / (1.f + nz);
        R[0] = fmaf(-nx * nx, f, 1.f); R[1] = -nx * ny * f;           R[2] = -nx;
        R[3] = -nx * ny * f;           R[4] = fmaf(-ny * ny, f, 1.f); R[5] = -ny;
        R[6] = nx;                     R[7] = ny;                     R[8] = nz;
    }

    for (int it = 0; ok && it < cfg.T; it++) {
        Coef k;
        k.cx0 = R[0] * cam.ifx; k.cy0 = R[1] * cam.ify;
        k.bx = fmaf(k.cx0, ap, fmaf(k.cy0, bp, R[2]));
        k.cx1 = R[3] * cam.ifx; k.cy1 = R[4] * cam.ify;
        k.by = fmaf(k.cx1, ap, fmaf(k.cy1, bp, R[5]));
        k.cx2 = R[6] * cam.ifx; k.cy2 = R[7] * cam.ify;
        k.bh = fmaf(k.cx2, ap, fmaf(k.cy2, bp, R[8]));
        k.A = A; k.B = B; k.C = C; k.tz = tz;
        k.hA = 0.5f * A; k.hC = 0.5f * C;
        k.invk = cfg.invk; k.Zp = Zp;

        float thr = 0.f;
        if (REJECT) {
            // MSE of the window at this iteration; keep eps^2 <= ratio * MSE
            float se = 0.f;
            int cnt = 0;
            for (int dv = -r0; dv <= r; dv += s) {
                const float2* row = ctr + dv * SW;
                const float fdv = (float)dv;
                const float rx = fdv * k.cy0, ry = fdv * k.cy1, rh = fdv * k.cy2;
                for (int du = -r0; du <= r; du += s) {
                    const float2 e = row[du];
                    se += sq_residual(k, e.x, e.y, (float)du, rx, ry, rh);
                    cnt += e.y == 1.f;
                }
            }
            thr = cfg.reject_ratio * (se / (float)cnt);
        }

        Moments m;
        zero(m);
        for (int dv = -r0; dv <= r; dv += s) {
            const float2* row = ctr + dv * SW;
            const float fdv = (float)dv;
            const float rx = fdv * k.cy0, ry = fdv * k.cy1, rh = fdv * k.cy2;
            if (RW > 0) {
#pragma unroll
                for (int du = -RW; du <= RW; du++) {
                    const float2 e = row[du];
                    visit<REJECT>(m, k, e.x, e.y, (float)du, rx, ry, rh, thr);
                }
            } else {
                for (int du = -r0; du <= r; du += s) {
                    const float2 e = row[du];
                    visit<REJECT>(m, k, e.x, e.y, (float)du, rx, ry, rh, thr);
                }
            }
        }

        float dl[6];
        if (!solve_update(m, cfg.pivot_tol, dl)) {
            ok = false;
            break;
        }
        rotate_left(R, dl[0], dl[1]);
        tz += dl[2];
        A += dl[3];
        B += dl[4];
        C += dl[5];
    }

    if (!ok) {
        k1o[out] = qnan();
        k2o[out] = qnan();
        if (nrmo) {
            nrmo[3 * out] = qnan();
            nrmo[3 * out + 1] = qnan();
            nrmo[3 * out + 2] = qnan();
        }
        return;
    }
    // ---- principal curvatures (Sec. 3.1.2) and refined normal (Sec. 3.2.4)
    const float T1 = 0.5f * (A + C);
    const float hd = 0.5f * (A - C);
    const float T2 = sqrtf(fmaf(hd, hd, B * B));
    k1o[out] = T1 + T2;
    k2o[out] = T1 - T2;
    if (nrmo) {
        nrmo[3 * out] = R[6];
        nrmo[3 * out + 1] = R[7];
        nrmo[3 * out + 2] = R[8];
    }
}

template <int RW>
cudaError_t launch_fit_rw(const float* depth, int H, int W, const Camera& cam, const FitConfig& cfg,
                          float* k1, float* k2, float* normal, cudaStream_t stream) {
    const dim3 block(TILE_W, TILE_H);
    const dim3 grid((W + TILE_W - 1) / TILE_W, (H + TILE_H - 1) / TILE_H);
    const size_t smem = fit_smem_bytes(cfg);
    if (cfg.reject)
        k_fit<RW, true><<<grid, block, smem, stream>>>(depth, H, W, cam, cfg, k1, k2, normal);
    else
        k_fit<RW, false><<<grid, block, smem, stream>>>(depth, H, W, cam, cfg, k1, k2, normal);
    return cudaGetLastError();
}

}  // namespace pcurv
