// pc_fit.cuh -- the fused per-pixel curvature kernel (sm_103a).
//
// One CTA computes a 32 x th tile of output pixels (th = 8 or 4 with one
// thread per pixel; th = 4, 2, 1 with lane groups of 2, 4, 8 per pixel).  The
// CTA first stages the tile's range values plus a halo of max(r, r_n) pixels
// into shared memory as two planes, Z and c, c = 1 for a valid range and +inf
// for none (outside the image, zero, negative or not finite), and counts the
// valid window points of every pixel row by row.  Each thread then runs the
// whole method of Spek, Li and Drummond (arXiv 1707.00385, Sec. 3.2) for its
// pixel in registers:
//
//   initial normal   Sec. 3.2.1, Eq. initialnormal (7x7 regression)
//   frame            Sec. 3.2.2 (minimal rotation to the normal, A=B=C=t_z=0)
//   T iterations     Sec. 3.2.3: residuals of Eq. quad, Jacobian, weights of
//                    Eq. weighting_function, the 6x6 system of
//                    Eq. iter_reweighted_update solved by an LDL^T
//                    factorisation judged on its Jacobi-scaled pivots,
//                    Gauss-Newton update
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
//   * window points are visited in pairs, p'(du, dv) with p'(-du, -dv), in
//     packed FP32x2 instructions (pc_f32x2.cuh): both points share every
//     per-iteration coefficient, their alpha coefficients are exact negatives
//     of each other, so one instruction does the work of two and each sum is
//     kept as a pair of partial sums, added once per iteration.  The centre
//     point (p' = 0) contributes only to sum w and sum w eps.
//   * single-precision rounding of a running sum grows with the number of
//     terms already in it, so the one-thread kernels sum PC_FOLD_ROWS window
//     rows at a time into fresh registers and fold each such partial into a
//     running total in shared memory, for the 20 sums of J^T W J: each term
//     then meets a sum over a few rows instead of the whole window.
#pragma once
#include <cfloat>
#include <cuda_runtime.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pc_f32x2.cuh"
#include "pc_internal.h"

// Column unroll factor of the window loops of the fixed-radius kernels
// (0 = unroll the whole row) and the CTAs per SM the register budget targets.
#ifndef PC_COL_UNROLL
#define PC_COL_UNROLL 0
#endif
#ifndef PC_MIN_BLOCKS
#define PC_MIN_BLOCKS 2
#endif
// Window rows summed into registers between two folds of the J^T W J sums
// into their shared-memory totals (one-thread FP32 kernels; windows of at
// least 2 PC_FOLD_ROWS pairs of rows).  GB300, 640 x 480, r = 7, T = 5:
// folding every row, every 2 and every 3 rows costs 4.0, 2.7 and 1.8 % of the
// throughput; every 2 rows brings 0.934 of a Kinect-like crop's pixels within
// the parity tolerance against 0.919 unfolded (every row: 0.935).
#ifndef PC_FOLD_ROWS
#define PC_FOLD_ROWS 3
#endif
#define PC_STR(x) #x
#define PC_UNROLL(n) _Pragma(PC_STR(unroll n))

namespace pcurv {

__device__ __forceinline__ float rcp_approx(float x) {
    // PTX rcp.approx.ftz.f32: at most 1 ulp of error; rcp(+inf) = +0.
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fffffff); }

// 26 running sums of one iteration, each as a pair of partial sums (the two
// points of a symmetric pair).  j0 is carried negated (nj0 = -j0).
struct Moments2 {
    f32x2 h00, h01, h11;       // sum w j0 j0, -w j0 j1, w j1 j1
    f32x2 s0, s1;              // sum -w j0, w j1
    f32x2 h03, h04, h05;       // sum -w j0 x^2, -w j0 x y, -w j0 y^2
    f32x2 h13, h14, h15;       // sum w j1 x^2, w j1 x y, w j1 y^2
    f32x2 sw;                  // sum w
    f32x2 sxx, sxy, syy;       // sum w x^2, w x y, w y^2
    f32x2 m40, m31, m22, m13, m04;  // sum w x^4, w x^3 y, w x^2 y^2, w x y^3, w y^4
    f32x2 g0, g1, ge, g3, g4, g5;   // sum -w eps j0, w eps j1, w eps, w eps x^2, w eps x y, w eps y^2
};

// Per-iteration constants of one pixel, splat into pairs.  With sigma = 1/sqrt(k)
// the loop carries e = sigma eps (so the Cauchy weight is 1 / (1 + e^2)) and
// hs = (2 / sigma) h, so that one gradient serves residual and Jacobian:
//   ga = sigma/2 (A x + B y), gb = sigma/2 (B x + C y),
//   e  = ga x + gb y - sigma h - sigma t_z,
//   j1 = (A x + B y) h + x = ga hs + x,  -j0 = (B x + C y) h + y = gb hs + y.
struct Coef2 {
    f32x2 cx0, cx1, cx2;       // x = Z (du cx0 + dv cy0) + dZ bx, likewise y and hs
    f32x2 bx, by, bh;
    f32x2 ga, gb, gc;          // sigma/2 (A, B, C)
    f32x2 nhs;                 // -sigma^2 / 2: -sigma h = nhs hs
    f32x2 nts;                 // -sigma t_z
    f32x2 nzp;                 // -Z_p
};

__device__ __forceinline__ void zero(Moments2& m) {
    const f32x2 z = 0ull;
    m.h00 = m.h01 = m.h11 = m.s0 = m.s1 = z;
    m.h03 = m.h04 = m.h05 = m.h13 = m.h14 = m.h15 = z;
    m.sw = m.sxx = m.sxy = m.syy = z;
    m.m40 = m.m31 = m.m22 = m.m13 = m.m04 = z;
    m.g0 = m.g1 = m.ge = m.g3 = m.g4 = m.g5 = z;
}

// Local coordinates (x, y, hs) of a pair (hs = (2/sigma) h, from the scaled h row).
// DU = (du, -du); RX = (dv cy0, -dv cy0).
__device__ __forceinline__ void local_xyz2(const Coef2& k, f32x2 Z, f32x2 DU, f32x2 RX, f32x2 RY,
                                           f32x2 RH, f32x2& X, f32x2& Y, f32x2& Hh) {
    const f32x2 dZ = add2(Z, k.nzp);
    X = fma2(fma2(DU, k.cx0, RX), Z, mul2(k.bx, dZ));
    Y = fma2(fma2(DU, k.cx1, RY), Z, mul2(k.by, dZ));
    Hh = fma2(fma2(DU, k.cx2, RH), Z, mul2(k.bh, dZ));
}

// Precision variants of the kernels (template parameter PREC): bit 0 selects
// compensated sums, bits 1-2 the range storage (0 float32, 1 FP16 offsets,
// 2 BF16 offsets from a per-tile base).
constexpr int PREC_KAHAN = 1;
__host__ __device__ constexpr int prec_format(int prec) { return prec >> 1; }

// sum += a * b, plain or compensated.  The compensated form (Kahan) keeps
// nc = -(rounding error so far): y = a b - c, t = s + y, c' = (t - s) - y.
template <bool KAHAN>
__device__ __forceinline__ void acc_fma(f32x2& s, f32x2& nc, f32x2 a, f32x2 b) {
    if (KAHAN) {
        const f32x2 y = fma2(a, b, nc);
        const f32x2 t = add2(s, y);
        nc = sub2(y, sub2(t, s));
        s = t;
    } else {
        s = fma2(a, b, s);
    }
}

template <bool KAHAN>
__device__ __forceinline__ void acc_add(f32x2& s, f32x2& nc, f32x2 x) {
    if (KAHAN) {
        const f32x2 y = add2(x, nc);
        const f32x2 t = add2(s, y);
        nc = sub2(y, sub2(t, s));
        s = t;
    } else {
        s = add2(s, x);
    }
}

// Scaled residuals e = sigma eps of a pair (with x, y, hs).
__device__ __forceinline__ f32x2 residual2(const Coef2& k, f32x2 X, f32x2 Y, f32x2 Hs, f32x2& GA,
                                          f32x2& GB) {
    GA = fma2(k.ga, X, mul2(k.gb, Y));
    GB = fma2(k.gb, X, mul2(k.gc, Y));
    return fma2(GA, X, fma2(GB, Y, fma2(k.nhs, Hs, k.nts)));
}

// One symmetric pair: residuals (the quadric of Sec. 3.2 in the local frame),
// Cauchy weights, Jacobian rows and the 26 sums (the eps sums scaled by sigma).
// C = (c_a, c_b), 1 valid / +inf invalid.  thr bounds e^2 when REJECT.
// c holds the compensations of the sums when KAHAN (unused otherwise).
// FIRST: the first iteration, where A = B = C = 0, so that e = -sigma (h + t_z),
// j1 = x, -j0 = y, and five sums repeat others (first_iteration_sums fills them).
template <bool REJECT, bool KAHAN, bool FIRST>
__device__ __forceinline__ void visit2(Moments2& m, Moments2& c, const Coef2& k, float za, float zb,
                                       float ca, float cb, f32x2 DU, f32x2 RX, f32x2 RY, f32x2 RH,
                                       float thr) {
    f32x2 X, Y, Hs, GA, GB;
    local_xyz2(k, pack(za, zb), DU, RX, RY, RH, X, Y, Hs);
    const f32x2 E = FIRST ? fma2(k.nhs, Hs, k.nts) : residual2(k, X, Y, Hs, GA, GB);
    float da, db;
    unpack(fma2(E, E, pack(ca, cb)), da, db);
    float wa = rcp_approx(da), wb = rcp_approx(db);
    if (REJECT) {
        float ea, eb;
        unpack(mul2(E, E), ea, eb);
        wa = ea <= thr ? wa : 0.f;
        wb = eb <= thr ? wb : 0.f;
    }
    const f32x2 Wt = pack(wa, wb);
    const f32x2 NJ0 = FIRST ? Y : fma2(GB, Hs, Y);
    const f32x2 J1 = FIRST ? X : fma2(GA, Hs, X);
    const f32x2 XX = mul2(X, X), XY = mul2(X, Y), YY = mul2(Y, Y);
    const f32x2 WE = mul2(Wt, E), WJ0 = mul2(Wt, NJ0), WJ1 = mul2(Wt, J1);
    const f32x2 WXX = mul2(Wt, XX), WYY = mul2(Wt, YY);
    // The sums are ordered so that each multiply-add shares an operand with the
    // one before it: a packed FMA whose three operands are all fresh registers
    // issues at about 0.7 of the FP32 rate, one with a repeated operand at ~0.9.
    acc_add<KAHAN>(m.s0, c.s0, WJ0);
    acc_add<KAHAN>(m.s1, c.s1, WJ1);
    acc_add<KAHAN>(m.sw, c.sw, Wt);
    acc_add<KAHAN>(m.sxx, c.sxx, WXX);
    acc_add<KAHAN>(m.syy, c.syy, WYY);
    acc_add<KAHAN>(m.ge, c.ge, WE);
    if (!FIRST) {
        // with j1 = x, -j0 = y these are sum w y^2, w x y, w x^2, w x^2 y, w x y^2
        acc_fma<KAHAN>(m.h00, c.h00, WJ0, NJ0);
        acc_fma<KAHAN>(m.h01, c.h01, WJ0, J1);
    }
    acc_fma<KAHAN>(m.h03, c.h03, WJ0, XX);
    acc_fma<KAHAN>(m.h04, c.h04, WJ0, XY);
    acc_fma<KAHAN>(m.h05, c.h05, WJ0, YY);
    if (!FIRST) {
        acc_fma<KAHAN>(m.h15, c.h15, WJ1, YY);
        acc_fma<KAHAN>(m.h14, c.h14, WJ1, XY);
    }
    acc_fma<KAHAN>(m.h13, c.h13, WJ1, XX);
    if (!FIRST) acc_fma<KAHAN>(m.h11, c.h11, WJ1, J1);
    acc_fma<KAHAN>(m.g1, c.g1, WE, J1);
    acc_fma<KAHAN>(m.g0, c.g0, WE, NJ0);
    acc_fma<KAHAN>(m.g3, c.g3, WE, XX);
    acc_fma<KAHAN>(m.g4, c.g4, WE, XY);
    acc_fma<KAHAN>(m.g5, c.g5, WE, YY);
    acc_fma<KAHAN>(m.m04, c.m04, WYY, YY);
    acc_fma<KAHAN>(m.m13, c.m13, WYY, XY);
    acc_fma<KAHAN>(m.sxy, c.sxy, Wt, XY);
    acc_fma<KAHAN>(m.m31, c.m31, WXX, XY);
    acc_fma<KAHAN>(m.m40, c.m40, WXX, XX);
    acc_fma<KAHAN>(m.m22, c.m22, WXX, YY);
}

// The sums the first iteration does not accumulate: with j1 = x and -j0 = y,
// sum w j0 j0 = sum w y^2, -sum w j0 j1 = sum w x y, sum w j1 j1 = sum w x^2,
// sum w j1 x y = -sum w j0 x^2 (negated convention: h03), sum w j1 y^2 = h04.
__device__ __forceinline__ void first_iteration_sums(Moments2& m, Moments2& c) {
    m.h00 = m.syy; m.h01 = m.sxy; m.h11 = m.sxx; m.h14 = m.h03; m.h15 = m.h04;
    c.h00 = c.syy; c.h01 = c.sxy; c.h11 = c.sxx; c.h14 = c.h03; c.h15 = c.h04;
}

// The 20 sums of J^T W J in the order of their shared-memory totals: total i
// of the thread lives at tot[i * nt] (nt = threads of the CTA, so a warp's
// 8-byte accesses are contiguous).  The first iteration accumulates only the
// first 15 (first_iteration_sums fills the other five from them).
#define PC_FOLD_FIRST(X) X(0, s0) X(1, s1) X(2, h03) X(3, h04) X(4, h05) X(5, h13) X(6, sw) X(7, sxx) \
    X(8, sxy) X(9, syy) X(10, m40) X(11, m31) X(12, m22) X(13, m13) X(14, m04)
#define PC_FOLD_LATER(X) X(15, h00) X(16, h01) X(17, h11) X(18, h14) X(19, h15)
static_assert(FOLD_SUMS == 20, "PC_FOLD_FIRST and PC_FOLD_LATER list the folded sums");

// total = the partial sums of the first rows; partial = 0
template <bool FIRST>
__device__ __forceinline__ void fold_start(Moments2& m, f32x2* tot, int nt) {
#define PC_FOLD_ONE(i, f) \
    tot[(i) * nt] = m.f; \
    m.f = 0ull;
    PC_FOLD_FIRST(PC_FOLD_ONE)
    if (!FIRST) { PC_FOLD_LATER(PC_FOLD_ONE) }
#undef PC_FOLD_ONE
}

// total += the partial sums of the rows since the last fold; partial = 0
template <bool FIRST>
__device__ __forceinline__ void fold_rows(Moments2& m, f32x2* tot, int nt) {
#define PC_FOLD_ONE(i, f) \
    tot[(i) * nt] = add2(tot[(i) * nt], m.f); \
    m.f = 0ull;
    PC_FOLD_FIRST(PC_FOLD_ONE)
    if (!FIRST) { PC_FOLD_LATER(PC_FOLD_ONE) }
#undef PC_FOLD_ONE
}

// partial sums of the last rows += their totals (the whole window's sums)
template <bool FIRST>
__device__ __forceinline__ void fold_finish(Moments2& m, const f32x2* tot, int nt) {
#define PC_FOLD_ONE(i, f) m.f = add2(m.f, tot[(i) * nt]);
    PC_FOLD_FIRST(PC_FOLD_ONE)
    if (!FIRST) { PC_FOLD_LATER(PC_FOLD_ONE) }
#undef PC_FOLD_ONE
}

// Squared scaled residuals e^2 of a pair, 0 for invalid points (rejection pre-pass).
__device__ __forceinline__ float sq_residual2(const Coef2& k, float za, float zb, float ca,
                                              float cb, f32x2 DU, f32x2 RX, f32x2 RY, f32x2 RH) {
    f32x2 X, Y, Hs, GA, GB;
    local_xyz2(k, pack(za, zb), DU, RX, RY, RH, X, Y, Hs);
    const f32x2 E = residual2(k, X, Y, Hs, GA, GB);
    float ea, eb;
    unpack(mul2(E, E), ea, eb);
    return (ca == 1.f ? ea : 0.f) + (cb == 1.f ? eb : 0.f);
}

// 1/x: hardware approximation in single precision (at most 1 ulp: PTX
// rcp.approx), correctly rounded in double.  mul_rn / fma_rn: one rounding
// each, written out so that no compiler contraction can differ between the
// kernels that inline the solve (their results must agree bit for bit).
__device__ __forceinline__ float inv(float x) {
    float y;
    asm("rcp.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ double inv(double x) { return 1.0 / x; }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// LDL^T solve of H b = g (H symmetric, upper triangle used), returning
// delta = -b.  The factorisation is judged on the pivots of the Jacobi-scaled
// matrix D H D, D = diag(H)^(-1/2), without forming it: D H D = (D L D^-1)
// (D d D) (D L D^-1)^T, so its pivots are d_j / H_jj, and LDL^T without
// pivoting has the same relative rounding errors on H as on D H D.
//   ok:  every H_jj > 0 and every d_j > tol H_jj (a NaN fails)
//   low: some d_j < low_tol H_jj or is NaN (the FP64 refactorisation test)
// With M_jk = L_jk d_k:  d_j = H_jj - sum_k L_jk M_jk,
// L_ij = (H_ji - sum_k L_ik M_jk) / d_j.  T is float or double.
template <typename T>
__device__ __forceinline__ void ldlt6(const T (&H)[6][6], const T (&g)[6], T delta[6], T tol, T low_tol, bool& ok,
                                      bool& low) {
    T L[6][6], M[6][6], d[6], id[6];
    bool good = true, under = false;
#pragma unroll
    for (int j = 0; j < 6; j++) {
#pragma unroll
        for (int k = 0; k < j; k++) M[j][k] = mul_rn(L[j][k], d[k]);
        T dj = H[j][j];
#pragma unroll
        for (int k = 0; k < j; k++) dj = fma_rn(-L[j][k], M[j][k], dj);
        good = good & (H[j][j] > T(0)) & (dj > mul_rn(tol, H[j][j]));
        under = under | !(dj >= mul_rn(low_tol, H[j][j]));
        d[j] = dj;
        id[j] = inv(dj);
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            T s = H[j][i];
#pragma unroll
            for (int k = 0; k < j; k++) s = fma_rn(-L[i][k], M[j][k], s);
            L[i][j] = mul_rn(s, id[j]);
        }
    }
    T z[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        T s = g[i];
#pragma unroll
        for (int k = 0; k < i; k++) s = fma_rn(-L[i][k], z[k], s);
        z[i] = s;
    }
#pragma unroll
    for (int i = 0; i < 6; i++) z[i] = mul_rn(z[i], id[i]);
#pragma unroll
    for (int i = 5; i >= 0; i--) {
        T s = z[i];
#pragma unroll
        for (int k = i + 1; k < 6; k++) s = fma_rn(-L[k][i], z[k], s);
        delta[i] = -s;
        z[i] = s;
    }
    ok = good;
    low = under;
}

// Folds the 26 pairs (with their compensations when KAHAN), adds the centre
// point (w_c to sum w, w_c eps_c to sum w eps), assembles J^T W J and J^T W eps
// and solves for the update delta = -b.  Singular when a diagonal entry is
// <= 0 or a scaled pivot is <= pivot_tol; with fp64_pivot > 0 a system whose
// smallest FP32 scaled pivot is below fp64_pivot is factorised again in FP64
// and judged on the FP64 pivots.
template <bool KAHAN>
__device__ __forceinline__ bool solve_update(const Moments2& m, const Moments2& c, float wc, float ec,
                                             float isig, float pivot_tol, float fp64_pivot,
                                             float delta[6]) {
#define PC_FOLD(f) (KAHAN ? hsum(add2(m.f, c.f)) : hsum(m.f))
    const float h00 = PC_FOLD(h00), h01 = -PC_FOLD(h01), h11 = PC_FOLD(h11);
    const float s0 = PC_FOLD(s0), s1 = PC_FOLD(s1);
    const float h03 = -PC_FOLD(h03), h04 = -PC_FOLD(h04), h05 = -PC_FOLD(h05);
    const float h13 = PC_FOLD(h13), h14 = PC_FOLD(h14), h15 = PC_FOLD(h15);
    const float sw = PC_FOLD(sw) + wc;
    const float sxx = PC_FOLD(sxx), sxy = PC_FOLD(sxy), syy = PC_FOLD(syy);
    const float m40 = PC_FOLD(m40), m31 = PC_FOLD(m31), m22 = PC_FOLD(m22), m13 = PC_FOLD(m13),
                m04 = PC_FOLD(m04);
    // the eps sums carry sigma = 1/sqrt(k): isig = sqrt(k) restores them
    const float g0 = -PC_FOLD(g0) * isig, g1 = PC_FOLD(g1) * isig, ge = fmaf(wc, ec, PC_FOLD(ge) * isig);
    const float g3 = PC_FOLD(g3) * isig, g4 = PC_FOLD(g4) * isig, g5 = PC_FOLD(g5) * isig;
#undef PC_FOLD
    float H[6][6];
    H[0][0] = h00; H[0][1] = h01; H[0][2] = s0;
    H[0][3] = 0.5f * h03; H[0][4] = h04; H[0][5] = 0.5f * h05;
    H[1][1] = h11; H[1][2] = -s1;
    H[1][3] = 0.5f * h13; H[1][4] = h14; H[1][5] = 0.5f * h15;
    H[2][2] = sw; H[2][3] = -0.5f * sxx; H[2][4] = -sxy; H[2][5] = -0.5f * syy;
    H[3][3] = 0.25f * m40; H[3][4] = 0.5f * m31; H[3][5] = 0.25f * m22;
    H[4][4] = m22; H[4][5] = 0.5f * m13;
    H[5][5] = 0.25f * m04;
    const float g[6] = {g0, g1, -ge, 0.5f * g3, g4, 0.5f * g5};
    bool ok, low;
    ldlt6<float>(H, g, delta, pivot_tol, fp64_pivot, ok, low);
    bool diag_pos = true;
#pragma unroll
    for (int i = 0; i < 6; i++) diag_pos = diag_pos & (H[i][i] > 0.f);
    if (fp64_pivot > 0.f && diag_pos && low) {
        double Hd[6][6], gd[6], dd[6];
#pragma unroll
        for (int i = 0; i < 6; i++) {
            gd[i] = g[i];
#pragma unroll
            for (int j = i; j < 6; j++) Hd[i][j] = H[i][j];
        }
        bool okd, lowd;
        ldlt6<double>(Hd, gd, dd, (double)pivot_tol, 0.0, okd, lowd);
#pragma unroll
        for (int i = 0; i < 6; i++) delta[i] = (float)dd[i];
        return okd;
    }
    return ok;
}

// R <- Rot(t0, t1, 0) R, Rot the rotation by angle |t| about t/|t|
// (Rodrigues: I + sin(th)/th [t]x + (1 - cos th)/th^2 [t]x^2).
// Gauss-Newton steps turn the frame by small angles, so both coefficients are
// taken from their Maclaurin series in th^2 while th <= 1/2:
//   sin(th)/th         = sum (-1)^n th^2n / (2n+1)!
//   (1 - cos th)/th^2  = sum (-1)^n th^2n / (2n+2)!
// through th^8; the first omitted terms are below 2.5e-11 there, far under
// single-precision rounding.  Larger angles use sincosf.
__device__ __forceinline__ void rotate_left(float R[9], float t0, float t1) {
    const float th2 = fmaf(t0, t0, t1 * t1);
    float sa, c1;
    if (th2 <= 0.25f) {
        sa = fmaf(fmaf(fmaf(fmaf(th2, 1.f / 362880.f, -1.f / 5040.f), th2, 1.f / 120.f), th2, -1.f / 6.f), th2,
                  1.f);
        c1 = fmaf(fmaf(fmaf(fmaf(th2, 1.f / 3628800.f, -1.f / 40320.f), th2, 1.f / 720.f), th2, -1.f / 24.f),
                  th2, 0.5f);
    } else {
        const float th = sqrtf(th2);
        float s, c;
        sincosf(0.5f * th, &s, &c);
        sa = 2.f * s * c / th;
        c1 = 2.f * s * s / th2;
    }
    const float c1t0 = mul_rn(c1, t0), c1t1 = mul_rn(c1, t1), c01 = mul_rn(c1t0, t1);
    const float q[9] = {fma_rn(-c1t1, t1, 1.f), c01,                    mul_rn(sa, t1),
                        c01,                    fma_rn(-c1t0, t0, 1.f), -mul_rn(sa, t0),
                        -mul_rn(sa, t1),        mul_rn(sa, t0),         fma_rn(-c1, th2, 1.f)};
    float o[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++)
            o[3 * i + j] = fmaf(q[3 * i], R[j], fmaf(q[3 * i + 1], R[3 + j], q[3 * i + 2] * R[6 + j]));
#pragma unroll
    for (int i = 0; i < 9; i++) R[i] = o[i];
}

// Visits every symmetric pair of the window of the thread's pixel once.
// zc, cc point at the pixel's own entries of the Z and c planes (row stride SW).
// Rows dv = -r0 .. -s pair with rows -dv; the centre row pairs du < 0 with -du.
// RW > 0: radius RW and stride RS fixed at compile time (columns unrolled).
// row_end(k) is called after the k-th pair of rows (k = 0, 1, ...), not after
// the centre row.
template <int RW, int RS = 1, typename F, typename E>
__device__ __forceinline__ void for_each_pair(const float* zc, const float* cc, int SW, int r, int s,
                                              F&& f, E&& row_end) {
    constexpr int R0 = RW > 0 ? (RW / RS) * RS : 0;  // largest sampled offset, compile-time form
    const int r0 = (r / s) * s;
    const f32x2 STEP = pack((float)s, -(float)s);
    int row = 0;
    for (int dv = -r0; dv < 0; dv += s, row++) {
        const float *za = zc + dv * SW, *zb = zc - dv * SW;
        const float *ca = cc + dv * SW, *cb = cc - dv * SW;
        const f32x2 DV = pack((float)dv, -(float)dv);
        f32x2 DU = pack(-(float)r0, (float)r0);
        if (RW > 0) {
#if PC_COL_UNROLL > 0
            PC_UNROLL(PC_COL_UNROLL)
#else
#pragma unroll
#endif
            for (int du = -R0; du <= R0; du += RS) {
                f(za[du], zb[-du], ca[du], cb[-du], DU, DV);
                DU = add2(DU, STEP);
            }
        } else {
            for (int du = -r0; du <= r0; du += s) {
                f(za[du], zb[-du], ca[du], cb[-du], DU, DV);
                DU = add2(DU, STEP);
            }
        }
        row_end(row);
    }
    const f32x2 DV0 = 0ull;
    f32x2 DU = pack(-(float)r0, (float)r0);
    if (RW > 0) {
#if PC_COL_UNROLL > 0
        PC_UNROLL(PC_COL_UNROLL)
#else
#pragma unroll
#endif
        for (int du = -R0; du < 0; du += RS) {
            f(zc[du], zc[-du], cc[du], cc[-du], DU, DV0);
            DU = add2(DU, STEP);
        }
    } else {
        for (int du = -r0; du < 0; du += s) {
            f(zc[du], zc[-du], cc[du], cc[-du], DU, DV0);
            DU = add2(DU, STEP);
        }
    }
}

template <int RW, int RS = 1, typename F>
__device__ __forceinline__ void for_each_pair(const float* zc, const float* cc, int SW, int r, int s, F&& f) {
    for_each_pair<RW, RS>(zc, cc, SW, r, s, f, [](int) {});
}

// The share of one lane of a group of G lanes that computes one pixel
// together: the window splits into row units, units 0 .. r0/s - 1 being the
// rows dv = -r0 + k s (each point paired with its reflection (-du, -dv)) and
// the last unit the centre row (du < 0 paired with -du); lane `sub` visits
// units sub, sub + G, ...  Every lane runs the same number of units and the
// same columns, so the group never diverges: a unit past the last is visited
// with every point masked, and so are the centre row's columns du >= 0
// (masked: c = +inf, weight exactly 0).
template <int RW, int G, typename F>
__device__ __forceinline__ void for_each_pair_lanes(const float* zc, const float* cc, int SW, int r, int s, int sub,
                                                    F&& f) {
    const int r0 = (r / s) * s;
    const int units = r0 / s + 1;
    const int per_lane = RW > 0 ? (RW + G) / G : (units + G - 1) / G;
    const float INF = __int_as_float(0x7f800000);
    const f32x2 STEP = pack((float)s, -(float)s);
#pragma unroll
    for (int ui = 0; ui < per_lane; ui++) {
        const int k = sub + ui * G;
        const bool live = k < units, centre = k == units - 1;
        const int dv = live ? -r0 + k * s : 0;
        const float *za = zc + dv * SW, *zb = zc - dv * SW;
        const float *ca = cc + dv * SW, *cb = cc - dv * SW;
        const f32x2 DV = pack((float)dv, -(float)dv);
        f32x2 DU = pack(-(float)r0, (float)r0);
        if (RW > 0) {
#pragma unroll
            for (int du = -RW; du <= RW; du++) {
                const bool off = !live || (centre && du >= 0);
                f(za[du], zb[-du], off ? INF : ca[du], off ? INF : cb[-du], DU, DV);
                DU = add2(DU, STEP);
            }
        } else {
            for (int du = -r0; du <= r0; du += s) {
                const bool off = !live || (centre && du >= 0);
                f(za[du], zb[-du], off ? INF : ca[du], off ? INF : cb[-du], DU, DV);
                DU = add2(DU, STEP);
            }
        }
    }
}

// Sum of v over the G adjacent lanes of a group (butterfly).  Every lane ends
// with the same bits: each step adds the same two numbers in every lane.
template <int G>
__device__ __forceinline__ float lane_group_sum(float v) {
#pragma unroll
    for (int o = 1; o < G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Folds each of the 26 pairs and sums it over the lane group (the second half
// of each pair is left 0, so the solve's own fold returns the group total).
template <int G>
__device__ __forceinline__ void reduce_lanes(Moments2& m) {
#define PC_GROUP(f) m.f = pack(lane_group_sum<G>(hsum(m.f)), 0.f);
    PC_GROUP(h00) PC_GROUP(h01) PC_GROUP(h11) PC_GROUP(s0) PC_GROUP(s1)
    PC_GROUP(h03) PC_GROUP(h04) PC_GROUP(h05) PC_GROUP(h13) PC_GROUP(h14) PC_GROUP(h15)
    PC_GROUP(sw) PC_GROUP(sxx) PC_GROUP(sxy) PC_GROUP(syy)
    PC_GROUP(m40) PC_GROUP(m31) PC_GROUP(m22) PC_GROUP(m13) PC_GROUP(m04)
    PC_GROUP(g0) PC_GROUP(g1) PC_GROUP(ge) PC_GROUP(g3) PC_GROUP(g4) PC_GROUP(g5)
#undef PC_GROUP
}

// Initial normal of Sec. 3.2.1 (Eq. initialnormal): least squares z = a x + b y + c
// over the valid points of the (2 rn + 1)^2 patch around the pixel, then
// n = (-a, -b, 1) / sqrt(1 + a^2 + b^2).  The regression runs in pixel-scaled
// camera coordinates centred on the pixel's own point, exact in single
// precision: x' = fx x = du Z_i + (u0 - cx)(Z_i - Z_p), likewise y' = fy y,
// z' = Z_i - Z_p, so a = fx a', b = fy b'.  Symmetric points (du, dv) and
// (-du, -dv) share packed FP32x2 operations; the centre adds only to the
// count.  zc points at the pixel's entry of a staged Z plane (row stride SW)
// holding 0 where the range is not valid; the centre itself must be valid.
// Returns false when fewer than 3 points are valid or det M <= det_tol (tr M)^2
// (M in metric coordinates).
// RN > 0: patch radius fixed at compile time (loops unrolled); RN == 0: rn_rt.
// CONST_DU (RN > 0 only): each pair's column offsets are compile-time constants
// instead of one packed add per pair; the same values, so the same bits.  The
// normal field alone takes it (GB300, 4096 x 4096: 0.430 -> 0.417 ms); the
// fused kernel keeps the add, whose registers are all in use.
template <int RN, bool CONST_DU = false>
__device__ __forceinline__ bool initial_normal(const float* zc, int SW, int rn_rt, float ap, float bp, float Zp,
                                               const Camera& cam, float det_tol, float& nx, float& ny,
                                               float& nz) {
    const int rn = RN > 0 ? RN : rn_rt;
    f32x2 N = 0ull, SX = 0ull, SY = 0ull, SZ = 0ull, SXX = 0ull, SXY = 0ull, SYY = 0ull, SXZ = 0ull,
          SYZ = 0ull;
    const f32x2 AP = splat(ap), BP = splat(bp), NZP = splat(-Zp);
    const f32x2 STEP = pack(1.f, -1.f);
#pragma unroll
    for (int dv = -rn; dv <= 0; dv++) {
        const float* za = zc + dv * SW;
        const float* zb = zc - dv * SW;
        const f32x2 DV = pack((float)dv, -(float)dv);
        f32x2 DUi = pack(-(float)rn, (float)rn);
        const int last = dv < 0 ? rn : -1;
#pragma unroll
        for (int du = -rn; du <= last; du++) {
            const f32x2 DU = CONST_DU && RN > 0 ? pack((float)du, -(float)du) : DUi;
            const float a = za[du], b = zb[-du];
            const f32x2 Z = pack(a, b);  // 0 where invalid
            const f32x2 M = pack(a > 0.f ? 1.f : 0.f, b > 0.f ? 1.f : 0.f);
            // masked coordinates, exactly 0 for an invalid point (Z = 0, M = 0) and
            // the unmasked values otherwise: M (Z - Zp), du Z + ap M (Z - Zp), ...;
            // M^2 = M, so the products of masked coordinates are masked too
            const f32x2 MZ = fma2(M, NZP, Z);
            const f32x2 MX = fma2(DU, Z, mul2(AP, MZ));
            const f32x2 MY = fma2(DV, Z, mul2(BP, MZ));
            N = add2(N, M);
            SX = add2(SX, MX);
            SY = add2(SY, MY);
            SZ = add2(SZ, MZ);
            SXX = fma2(MX, MX, SXX);
            SXY = fma2(MX, MY, SXY);
            SXZ = fma2(MX, MZ, SXZ);
            SYY = fma2(MY, MY, SYY);
            SYZ = fma2(MY, MZ, SYZ);
            if (!(CONST_DU && RN > 0)) DUi = add2(DUi, STEP);
        }
    }
    const float n = hsum(N) + 1.f;  // + the centre, at x' = y' = z' = 0
    const float sx = hsum(SX), sy = hsum(SY), sz = hsum(SZ);
    const float sxx = hsum(SXX), sxy = hsum(SXY), syy = hsum(SYY), sxz = hsum(SXZ), syz = hsum(SYZ);
    // centred second moments M' and v' (shift by the centre point first)
    const float in = 1.f / n;
    const float mx = sx * in, my = sy * in, mz = sz * in;
    const float m00 = fmaf(-sx, mx, sxx), m01 = fmaf(-sx, my, sxy), m11 = fmaf(-sy, my, syy);
    const float w0 = fmaf(-sx, mz, sxz), w1 = fmaf(-sy, mz, syz);
    // the singularity test in metric coordinates: M = S M' S, S = diag(1/fx, 1/fy)
    const float ix2 = cam.ifx * cam.ifx, iy2 = cam.ify * cam.ify;
    const float det = fmaf(m00, m11, -m01 * m01) * (ix2 * iy2), tr = fmaf(m00, ix2, m11 * iy2);
    if (n < 3.f || !(det > det_tol * tr * tr)) return false;
    const float idet = 1.f / fmaf(m00, m11, -m01 * m01);
    const float a = mul_rn(mul_rn(fma_rn(m11, w0, -mul_rn(m01, w1)), idet), cam.fx);
    const float b = mul_rn(mul_rn(fma_rn(m00, w1, -mul_rn(m01, w0)), idet), cam.fy);
    const float sc = rsqrtf(fmaf(a, a, fmaf(b, b, 1.f)));
    nx = -a * sc;
    ny = -b * sc;
    nz = sc;
    return true;
}

// The whole method for one 32 x TH output tile (tile column tx_, tile row ty_)
// of frame f.  Called by every thread of the CTA (32 x TH G threads, TH G
// warps); contains one __syncthreads and leaves shared memory in use until it
// returns (callers that reuse smem synchronise first).
// RW > 0: window radius RW and sampling stride RS fixed at compile time,
// columns unrolled.  RW == 0: radius and stride from cfg.
// G: lanes per pixel.  G = 1: one thread per pixel.  G > 1: G adjacent lanes
// share a pixel's window rows (for_each_pair_lanes) and sum their moments
// (reduce_lanes) before each solve, which every lane of the group repeats;
// only the order of the moment sums differs from G = 1.
template <int RW, bool REJECT, int PREC = 0, int TH = 8, int G = 1, int RS = 1>
__device__ __forceinline__ void fit_tile(const FrameArgs& f, const FitConfig& cfg, int tx_, int ty_,
                                         float* smem) {
    constexpr bool KAHAN = (PREC & PREC_KAHAN) != 0;
    constexpr int FMT = prec_format(PREC);
    constexpr int NW = TH * G;  // warps of the CTA
    // fold the J^T W J sums row by row (one thread per pixel, plain sums)
    constexpr bool FOLD = G == 1 && !KAHAN;
    static_assert(G == 1 || G == 2 || G == 4 || G == 8, "lanes per pixel");
    static_assert(G == 1 || (!KAHAN && FMT == 0), "lane groups run the plain FP32 form");
    static_assert(G == 1 || RW == 0 || RS == 1, "lane groups with a compile-time window are dense");
    const float* __restrict__ depth = f.depth;
    const int H = f.H, W = f.W;
    const Camera cam = f.cam;
    float* __restrict__ k1o = f.k1;
    float* __restrict__ k2o = f.k2;
    float* __restrict__ nrmo = f.normal;
    const int r = RW > 0 ? RW : cfg.r;
    const int s = RW > 0 ? RS : cfg.stride;
    const int r0 = (r / s) * s;   // largest sampled offset
    const int halo = r > cfg.rn ? r : cfg.rn;
    const int SW = TILE_W + 2 * halo;
    const int SH = TH + 2 * halo;
    float* tz = smem;                       // Z plane, SH x SW
    float* tcv = smem + SW * SH;            // c plane
    int* rcnt = (int*)(tcv + SW * SH);      // valid window points per (tile row, pixel column)
    // folded totals: FOLD_SUMS pairs per thread after the planes (8-byte aligned)
    f32x2* fold_tot = (f32x2*)(smem + ((2 * SW * SH + SH * TILE_W + 1) & ~1)) +
                      (threadIdx.y * TILE_W + threadIdx.x);
    const int ub = tx_ * TILE_W, vb = ty_ * TH;

    // stage the tile + halo (Sec. 3.2, first item: the range image): warp w
    // takes halo rows w, w + NW, ..., its lanes the columns in passes of 32.
    // The validity bits of a row (ballots, SW <= 32 + 2 PC_MAX_RADIUS <= 96
    // columns) give the valid window points of every row segment
    // (columns -r0..r0 on the stride) by one population count per pixel column.
    unsigned long long seg = 0;  // the segment's sampled offsets as bits 0..2 r0
    if (s == 1) {
        seg = (2ull << (2 * r0)) - 1ull;
    } else {
        for (int k = 0; k <= 2 * r0; k += s) seg |= 1ull << k;
    }
    const int lane = threadIdx.x;
    for (int sy = threadIdx.y; sy < SH; sy += NW) {
        const int gv = vb - halo + sy;
        const bool row_in = gv >= 0 && gv < H;
        unsigned long long lo = 0, hi = 0;  // validity of columns 0..63, 64..95
#pragma unroll
        for (int pass = 0; pass < 3; pass++) {
            const int sx = pass * 32 + lane;
            if (pass * 32 >= SW) break;  // uniform over the warp
            const int gu = ub - halo + sx;
            float z = 0.f, c = __int_as_float(0x7f800000);
            if (sx < SW && row_in && gu >= 0 && gu < W) {
                float d;
                if (FMT == 0) {
                    d = __ldg(depth + (size_t)gv * W + gu);
                } else {
                    // centred 16-bit storage: range = tile base + offset
                    const unsigned short q = __ldg(f.packed + (size_t)gv * W + gu);
                    const float off = FMT == 1 ? __half2float(__ushort_as_half(q))
                                               : __bfloat162float(__ushort_as_bfloat16(q));
                    d = __ldg(f.tile_base + (size_t)(gv / PACK_TILE_H) * ((W + TILE_W - 1) / TILE_W) +
                              gu / TILE_W) +
                        off;
                }
                if (d > 0.f && d <= FLT_MAX) {
                    z = d;
                    c = 1.f;
                }
            }
            if (sx < SW) {
                tz[sy * SW + sx] = z;
                tcv[sy * SW + sx] = c;
            }
            const unsigned long long bits = __ballot_sync(0xffffffffu, c == 1.f);
            if (pass == 0) lo = bits;
            else if (pass == 1) lo |= bits << 32;
            else hi = bits;
        }
        // bits col + halo - r0 ... col + halo + r0 of the row: start <= 31 + halo <= 55
        const int start = lane + halo - r0;
        const unsigned long long w = (lo >> start) | (start > 0 ? hi << (64 - start) : 0ull);
        rcnt[sy * TILE_W + lane] = __popcll(w & seg);
    }
    __syncthreads();

    // the thread's pixel (tile column pxl, row pyl) and its lane in the group
    int pxl, pyl, sub = 0;
    if constexpr (G == 1) {
        pxl = threadIdx.x;
        pyl = threadIdx.y;
    } else {
        const int t = threadIdx.y * TILE_W + threadIdx.x;
        pxl = (t / G) % TILE_W;
        pyl = t / G / TILE_W;
        sub = t % G;
    }
    const int u0 = ub + pxl, v0 = vb + pyl;
    const bool inside = u0 < W && v0 < H;
    // no barrier follows in this function; lane groups keep every lane for
    // their shuffles (a pixel outside the image computes on staged values and
    // stores nothing)
    if constexpr (G == 1) {
        if (!inside) return;
    }
    const int cidx = (pyl + halo) * SW + pxl + halo;
    const float* zc = tz + cidx;
    const float* cc = tcv + cidx;
    const float Zp = *zc;
    const float ap = (float)u0 - cam.cx, bp = (float)v0 - cam.cy;
    bool ok = (G == 1 || inside) && *cc == 1.f;

    // ---- initial normal: z = a x + b y + c over the valid (2rn+1)^2 patch
    float nx = 0.f, ny = 0.f, nz = 1.f;
    if (ok)
        ok = cfg.rn == NORMAL_RADIUS_UNROLLED
                 ? initial_normal<NORMAL_RADIUS_UNROLLED>(zc, SW, 0, ap, bp, Zp, cam, cfg.det_tol, nx, ny, nz)
                 : initial_normal<0>(zc, SW, cfg.rn, ap, bp, Zp, cam, cfg.det_tol, nx, ny, nz);

    // ---- window count (row segments counted above)
    int cnt = 0;
    if (ok) {
        const int* rc = rcnt + (pyl + halo) * TILE_W + pxl;
        for (int dv = -r0; dv <= r0; dv += s) cnt += rc[dv * TILE_W];
        ok = cnt >= cfg.min_window;
    }

    float R[9];
    float A = 0.f, B = 0.f, C = 0.f, tz0 = 0.f;
    {
        // minimal rotation with R n = e_z: I + [w]x + [w]x^2/(1+n_z), w = n x e_z
        const float f = 1.f / (1.f + nz);
        R[0] = fmaf(-nx * nx, f, 1.f); R[1] = -nx * ny * f;           R[2] = -nx;
        R[3] = -nx * ny * f;           R[4] = fmaf(-ny * ny, f, 1.f); R[5] = -ny;
        R[6] = nx;                     R[7] = ny;                     R[8] = nz;
    }

    // sigma = 1/sqrt(k) scales the residuals carried by the loop (Coef2)
    const float sig = sqrtf(cfg.invk), isig = 1.f / sig, hscale = 2.f * isig;
    for (int it = 0; it < cfg.T; it++) {
        if constexpr (G == 1) {
            if (!ok) break;
        } else {
            if (!__any_sync(0xffffffffu, ok)) break;  // uniform over the warp
        }
        Coef2 k;
        const float cx0 = R[0] * cam.ifx, cy0 = R[1] * cam.ify;
        const float cx1 = R[3] * cam.ifx, cy1 = R[4] * cam.ify;
        const float cx2 = R[6] * cam.ifx, cy2 = R[7] * cam.ify;
        k.cx0 = splat(cx0); k.cx1 = splat(cx1); k.cx2 = splat(cx2 * hscale);
        k.bx = splat(fmaf(cx0, ap, fmaf(cy0, bp, R[2])));
        k.by = splat(fmaf(cx1, ap, fmaf(cy1, bp, R[5])));
        k.bh = splat(fmaf(cx2, ap, fmaf(cy2, bp, R[8])) * hscale);
        const float hsig = 0.5f * sig;
        k.ga = splat(hsig * A); k.gb = splat(hsig * B); k.gc = splat(hsig * C);
        k.nhs = splat(-0.5f * cfg.invk);
        k.nts = splat(-sig * tz0);
        k.nzp = splat(-Zp);
        const f32x2 CY0 = splat(cy0), CY1 = splat(cy1), CY2 = splat(cy2 * hscale);
        // the centre point: p' = 0, so eps_c = -t_z and j_c = (0, 0, -1, 0, 0, 0)
        const float ec = -tz0;
        const float wc = rcp_approx(fmaf(ec * ec, cfg.invk, 1.f));

        float thr = 0.f;
        if (REJECT) {
            // MSE of the window at this iteration; keep eps^2 <= ratio * MSE
            // (both sides in units of k: e^2 = eps^2 / k)
            float se = 0.f;
            auto sq = [&](float za, float zb, float ca, float cb, f32x2 DU, f32x2 DV) {
                se += sq_residual2(k, za, zb, ca, cb, DU, mul2(DV, CY0), mul2(DV, CY1), mul2(DV, CY2));
            };
            if constexpr (G == 1) {
                for_each_pair<RW, RS>(zc, cc, SW, r, s, sq);
            } else {
                for_each_pair_lanes<RW, G>(zc, cc, SW, r, s, sub, sq);
                se = lane_group_sum<G>(se);
            }
            const float esc = -sig * tz0;
            se += esc * esc;
            thr = cfg.reject_ratio * (se / (float)cnt);
        }
        const float esc2 = (sig * tz0) * (sig * tz0);
        const float wcr = (REJECT && !(esc2 <= thr)) ? 0.f : wc;

        Moments2 m, comp;
        zero(m);
        zero(comp);
        auto first = [&](float za, float zb, float ca, float cb, f32x2 DU, f32x2 DV) {
            visit2<REJECT, KAHAN, true>(m, comp, k, za, zb, ca, cb, DU, mul2(DV, CY0), mul2(DV, CY1),
                                        mul2(DV, CY2), thr);
        };
        auto later = [&](float za, float zb, float ca, float cb, f32x2 DU, f32x2 DV) {
            visit2<REJECT, KAHAN, false>(m, comp, k, za, zb, ca, cb, DU, mul2(DV, CY0), mul2(DV, CY1),
                                         mul2(DV, CY2), thr);
        };
        // fold the J^T W J partials after every PC_FOLD_ROWS pairs of rows: the
        // first fold starts the totals, the centre row's partial joins at the end
        constexpr int NT = TILE_W * TH;
        const bool folded = FOLD && r0 / s >= 2 * PC_FOLD_ROWS;
        auto fold_first = [&](int row) {
            if constexpr (FOLD) {
                if (!folded || (row + 1) % PC_FOLD_ROWS != 0) return;
                if (row + 1 == PC_FOLD_ROWS) fold_start<true>(m, fold_tot, NT);
                else fold_rows<true>(m, fold_tot, NT);
            }
        };
        auto fold_later = [&](int row) {
            if constexpr (FOLD) {
                if (!folded || (row + 1) % PC_FOLD_ROWS != 0) return;
                if (row + 1 == PC_FOLD_ROWS) fold_start<false>(m, fold_tot, NT);
                else fold_rows<false>(m, fold_tot, NT);
            }
        };
        if (it == 0) {
            // A = B = C = 0 here: the cheaper first-iteration form
            if constexpr (G == 1) {
                for_each_pair<RW, RS>(zc, cc, SW, r, s, first, fold_first);
                if (folded) fold_finish<true>(m, fold_tot, NT);
            } else {
                for_each_pair_lanes<RW, G>(zc, cc, SW, r, s, sub, first);
            }
            first_iteration_sums(m, comp);
        } else {
            if constexpr (G == 1) {
                for_each_pair<RW, RS>(zc, cc, SW, r, s, later, fold_later);
                if (folded) fold_finish<false>(m, fold_tot, NT);
            } else {
                for_each_pair_lanes<RW, G>(zc, cc, SW, r, s, sub, later);
            }
        }
        if constexpr (G > 1) reduce_lanes<G>(m);

        float dl[6];
        const bool solved = solve_update<KAHAN>(m, comp, wcr, ec, isig, cfg.pivot_tol, cfg.fp64_pivot, dl);
        if constexpr (G == 1) {
            if (!solved) {
                ok = false;
                break;
            }
        } else {
            ok = ok && solved;  // every lane of the group decides alike
            if (!ok) continue;
        }
        rotate_left(R, dl[0], dl[1]);
        tz0 += dl[2];
        A += dl[3];
        B += dl[4];
        C += dl[5];
    }

    if constexpr (G > 1) {
        if (sub != 0 || !inside) return;
    }
    const size_t out = (size_t)v0 * W + u0;
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

// Compensated sums need a pair of registers more per sum: those variants keep
// one CTA per SM instead of spilling.
#define PC_BLOCKS_OF(PREC) (((PREC) & PREC_KAHAN) ? 1 : PC_MIN_BLOCKS)

// One CTA per tile; grid row y computes tile row ty0 + y of the frame (a band
// of tile rows when ty0 > 0 or the grid is shorter than the frame).
template <int RW, bool REJECT, int PREC, int TH, int G, int RS>
__global__ void __launch_bounds__(TILE_W * TH * G, PC_BLOCKS_OF(PREC) * (8 / (TH * G)))
    k_fit(FrameArgs f, FitConfig cfg, int ty0) {
    extern __shared__ float smem[];
    fit_tile<RW, REJECT, PREC, TH, G, RS>(f, cfg, blockIdx.x, ty0 + blockIdx.y, smem);
}

// Persistent form over many frames: the CTAs take (frame, tile) items from a
// flattened queue until it is empty.  CTA b first takes item b -- the first
// CTAs of a launch are spread over the SMs, so a queue shorter than the grid
// still gets one item per SM -- then items gridDim.x, gridDim.x + 1, ... with
// one atomic each.  The header and descriptors live in device memory
// (BatchTable); *next_tile must be 0 at launch.
template <int RW, bool REJECT, int PREC, int TH, int G, int RS>
__global__ void __launch_bounds__(TILE_W * TH * G, PC_BLOCKS_OF(PREC) * (8 / (TH * G)))
    k_fit_batch(const BatchTable* __restrict__ table, unsigned* __restrict__ next_tile, FitConfig cfg) {
    extern __shared__ float smem[];
    __shared__ int s_tile;
    const int nframes = table->nframes, total = table->total_tiles;
    const BatchFrame* __restrict__ fr = table->frames;
    for (int t = blockIdx.x;;) {
        if (t >= total) break;  // uniform over the CTA
        // last frame whose first tile is <= t
        int lo = 0, hi = nframes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (fr[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
        }
        const int local = t - fr[lo].tile_begin, tiles_x = fr[lo].tiles_x;
        const int ty_ = local / tiles_x;
        fit_tile<RW, REJECT, PREC, TH, G, RS>(fr[lo].f, cfg, local - ty_ * tiles_x, ty_, smem);
        __syncthreads();  // shared memory and s_tile are reused by the next tile
        if (threadIdx.x == 0 && threadIdx.y == 0) s_tile = (int)(gridDim.x + atomicAdd(next_tile, 1u));
        __syncthreads();
        t = s_tile;
    }
}

// Dynamic shared memory of a kernel variant: planes, counts and, for the
// one-thread FP32 kernels, the folded totals of its 32 x TH threads.
template <int PREC, int TH, int G>
size_t variant_smem_bytes(const FitConfig& cfg) {
    constexpr bool FOLD = G == 1 && (PREC & PREC_KAHAN) == 0;
    return fit_smem_bytes(cfg, TH, FOLD ? TILE_W * TH : 0);
}

// Kernels whose dynamic shared memory exceeds the default 48 KB opt in on the
// current device (idempotent; needed before a launch or occupancy query).
template <typename K>
cudaError_t allow_smem(K kernel, size_t smem) {
    if (smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Tile rows ty0 .. ty1 - 1 of the frame (0 <= ty0 < ty1 <= its tile rows).
template <int RW, int PREC, int TH, int G = 1, int RS = 1>
cudaError_t launch_fit_rw(const FrameArgs& f, const FitConfig& cfg, cudaStream_t stream, int ty0, int ty1) {
    const dim3 block(TILE_W, TH * G);
    const dim3 grid((f.W + TILE_W - 1) / TILE_W, ty1 - ty0);
    const size_t smem = variant_smem_bytes<PREC, TH, G>(cfg);
    cudaError_t e;
    if (cfg.reject) {
        if ((e = allow_smem(k_fit<RW, true, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
        k_fit<RW, true, PREC, TH, G, RS><<<grid, block, smem, stream>>>(f, cfg, ty0);
    } else {
        if ((e = allow_smem(k_fit<RW, false, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
        k_fit<RW, false, PREC, TH, G, RS><<<grid, block, smem, stream>>>(f, cfg, ty0);
    }
    return cudaGetLastError();
}

template <int RW, int PREC, int TH, int G = 1, int RS = 1>
cudaError_t launch_batch_rw(const BatchTable* table, unsigned* next_tile, int grid, const FitConfig& cfg,
                            cudaStream_t stream) {
    const dim3 block(TILE_W, TH * G);
    const size_t smem = variant_smem_bytes<PREC, TH, G>(cfg);
    cudaError_t e;
    if (cfg.reject) {
        if ((e = allow_smem(k_fit_batch<RW, true, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
        k_fit_batch<RW, true, PREC, TH, G, RS><<<grid, block, smem, stream>>>(table, next_tile, cfg);
    } else {
        if ((e = allow_smem(k_fit_batch<RW, false, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
        k_fit_batch<RW, false, PREC, TH, G, RS><<<grid, block, smem, stream>>>(table, next_tile, cfg);
    }
    return cudaGetLastError();
}

template <int RW, int PREC, int TH, int G = 1, int RS = 1>
cudaError_t occupancy_rw(const FitConfig& cfg, int* blocks_per_sm) {
    const size_t smem = variant_smem_bytes<PREC, TH, G>(cfg);
    cudaError_t e;
    if (cfg.reject) {
        if ((e = allow_smem(k_fit_batch<RW, true, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fit_batch<RW, true, PREC, TH, G, RS>,
                                                             TILE_W * TH * G, smem);
    }
    if ((e = allow_smem(k_fit_batch<RW, false, PREC, TH, G, RS>, smem)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fit_batch<RW, false, PREC, TH, G, RS>,
                                                         TILE_W * TH * G, smem);
}

// The one-lane variants (32 x 8 and 32 x 4 tiles) of radius RW sampled every
// RS pixels (RW = 0: run-time radius and stride); the lane-group entries stay
// empty.
template <int RW, int PREC, int RS = 1>
const KernelOps* make_ops() {
    static const KernelOps k = {{launch_fit_rw<RW, PREC, 8, 1, RS>, launch_fit_rw<RW, PREC, 4, 1, RS>},
                                {launch_batch_rw<RW, PREC, 8, 1, RS>, launch_batch_rw<RW, PREC, 4, 1, RS>},
                                {occupancy_rw<RW, PREC, 8, 1, RS>, occupancy_rw<RW, PREC, 4, 1, RS>}};
    return &k;
}

// The lane-group variants of radius RW (FP32 ranges, plain sums): 32 x 4
// pixels with 2 lanes each, 32 x 2 with 4, 32 x 1 with 8 (256 threads each);
// the one-lane entries stay empty.
template <int RW>
const KernelOps* make_lane_ops() {
    static const KernelOps k = {
        {nullptr, nullptr, launch_fit_rw<RW, 0, 4, 2>, launch_fit_rw<RW, 0, 2, 4>, launch_fit_rw<RW, 0, 1, 8>},
        {nullptr, nullptr, launch_batch_rw<RW, 0, 4, 2>, launch_batch_rw<RW, 0, 2, 4>, launch_batch_rw<RW, 0, 1, 8>},
        {nullptr, nullptr, occupancy_rw<RW, 0, 4, 2>, occupancy_rw<RW, 0, 2, 4>, occupancy_rw<RW, 0, 1, 8>}};
    return &k;
}

}  // namespace pcurv
