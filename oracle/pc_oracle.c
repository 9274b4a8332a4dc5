/*
 * pc_oracle.c -- FP64 CPU oracle for dense per-pixel principal curvature from
 * a range image, after Spek, Li and Drummond, "A Fast Method For Computing
 * Principal Curvatures From Range Images" (arXiv 1707.00385).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark load this library. It shares no code, header,
 * table or constant with the CUDA path, and it never calls it.
 *
 * Everything is plain double precision, one pixel at a time, in the order of
 * the paper's pipeline (Sec. 3.2):
 *
 *   1. back-projection of the range image through the pinhole intrinsics
 *      (Sec. 3.2, first pipeline item; "range images" in Sec. 1);
 *   2. initial normal: z regressed linearly on x and y over a 7x7 patch,
 *      (a, b) = M^-1 v, n = (-a, -b, 1) / sqrt(1 + a^2 + b^2)
 *      (Sec. 3.2.1, Eq. initialnormal);
 *   3. frame R aligning the local z axis with that normal, A = B = C = t_z = 0
 *      (Sec. 3.2.2);
 *   4. per window point p'_i = p_i - p (Sec. 3.1.2), its residual
 *      eps_i = p~'^T E^T Q E p~' with E = [R | (0,0,t_z)] and the parabolic
 *      quadric Q(A, B, C) (Sec. 3.1.2, Eq. quad; Eq. error_func);
 *   5. the Jacobian of eps_i with respect to (theta_x, theta_y, t_z, A, B, C),
 *      formed from the derivatives of E and Q (Sec. 3.2.3);
 *   6. weights W(eps) = k / (k + eps^2), optionally zero when eps^2 exceeds
 *      R = ratio * MSE (Sec. 3.2.3, Eq. weighting_function);
 *   7. b = (J^T W J)^-1 J^T W eps (Sec. 3.2.3, Eq. iter_reweighted_update),
 *      applied as a Gauss-Newton step (parameters minus b);
 *   8. after the last iteration, T1 = (A + C)/2, T2 = sqrt(T1^2 - AC + B^2),
 *      k1 = T1 + T2, k2 = T1 - T2 (Sec. 3.1.2, closed form after Eq. quad);
 *   9. the refined normal is the final frame's local z axis (Sec. 3.2.4).
 *
 * Readings of the paper where it is silent or ambiguous (each one is listed in
 * the design notes of this repository):
 *   - x, y, z of the initial-normal regression are metric camera coordinates;
 *   - R is perturbed on the left by a rotation about the local x and y axes
 *     (theta_x, theta_y); the in-plane angle stays the one of the minimal
 *     rotation taking the initial normal to e_z;
 *   - Eq. iter_update is a Gauss-Newton step: parameters <- parameters - b;
 *   - the iteration count T is fixed, with no early exit;
 *   - the window is the dense (2r+1)^2 pixel square around the centre (or its
 *     points on a sampling stride), clipped to the image, including the
 *     centre; pixels without a valid range carry no weight;
 *   - with rejection, a point keeps its weight when eps^2 <= ratio * MSE, MSE
 *     being the mean of eps^2 over the window at the same iteration;
 *   - the validity rules below (det, pivot and count thresholds) are ours.
 *
 * Parity: pinned against closed forms, finite differences, least squares,
 * brute-force minimisation and brute-force window listing by the test suite.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EXPORT __attribute__((visibility("default")))

/* status codes of a pixel */
#define OR_OK 0
#define OR_INVALID_CENTRE 1 /* no valid range at the centre pixel */
#define OR_BAD_NORMAL 2     /* initial-normal regression degenerate */
#define OR_FEW_POINTS 3     /* fewer than min_window valid window points */
#define OR_SINGULAR 4       /* normal equations singular at some iteration */

typedef struct {
    double fx, fy, cx, cy; /* pinhole intrinsics in pixels; pixel centres at integer (u, v) */
    int r;                 /* fitting window radius: (2r+1)^2 patch */
    int rn;                /* initial-normal radius: (2rn+1)^2 patch, 3 gives 7x7 */
    int T;                 /* number of re-weighted iterations */
    int stride;            /* window sampling stride; 1 = dense */
    double k;              /* constant k of the weighting function */
    int reject;            /* 1 = rejection filter of the weighting function */
    double reject_ratio;   /* R = reject_ratio * MSE */
    double det_tol;        /* initial normal degenerate when det M <= det_tol (tr M)^2 */
    double pivot_tol;      /* normal equations singular when a scaled pivot <= pivot_tol */
    int min_window;        /* fewest valid window points accepted */
    double perturb;        /* sensitivity probe: relative noise on the normal equations and on
                              the initial-normal sums (0 = off) */
    double perturb_points; /* sensitivity probe: relative noise on each p' coordinate (0 = off) */
    unsigned long long perturb_seed;
    int f32_sums;          /* calibration of the probe, not the method: 1 = p' rounded to single
                              precision and every sum of the normal equations and of the
                              initial-normal regression added in single precision; 2, 3 = the
                              same with J^T W J from TF32 features (see normal_equations_f32) */
} or_params;

typedef struct {
    int status;
    int iters;           /* iterations completed */
    int npts;            /* valid window points */
    double k1, k2;       /* principal curvatures, k1 >= k2 */
    double normal[3];    /* refined normal (camera frame, unit, n_z > 0 at start) */
    double n0[3];        /* initial normal */
    double A, B, C, tz;  /* final quadric and offset */
    double R[9];         /* final rotation, row major, camera -> local */
    double min_pivot;    /* smallest scaled Cholesky pivot over all iterations */
    double last_b[6];    /* the update b of the last iteration (0 when T = 0) */
    double cond;         /* condition estimate: largest ratio of the largest to the smallest
                            scaled Cholesky pivot of one iteration, over all iterations */
} or_result;

/* ------------------------------------------------------------------------ */
/* small dense helpers (row-major)                                           */

static void mat4_mul(const double* a, const double* b, double* c) {
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double s = 0.0;
            for (int k = 0; k < 4; k++) s += a[4 * i + k] * b[4 * k + j];
            c[4 * i + j] = s;
        }
}

static void mat4_vec(const double* a, const double* x, double* y) {
    for (int i = 0; i < 4; i++) {
        double s = 0.0;
        for (int k = 0; k < 4; k++) s += a[4 * i + k] * x[k];
        y[i] = s;
    }
}

static double dot4(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

static void mat3_mul(const double* a, const double* b, double* c) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0.0;
            for (int k = 0; k < 3; k++) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

/* [w]_x, the cross-product matrix: [w]_x v = w x v */
static void skew(const double w[3], double S[9]) {
    S[0] = 0.0;   S[1] = -w[2]; S[2] = w[1];
    S[3] = w[2];  S[4] = 0.0;   S[5] = -w[0];
    S[6] = -w[1]; S[7] = w[0];  S[8] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* step 1: back-projection (Sec. 3.2, first pipeline item)                  */

static int range_valid(double z) { return z > 0.0 && isfinite(z); }

/* P = ((u - cx) z / fx, (v - cy) z / fy, z) */
OR_EXPORT void or_backproject(const or_params* p, int u, int v, double z, double P[3]) {
    P[0] = ((double)u - p->cx) * z / p->fx;
    P[1] = ((double)v - p->cy) * z / p->fy;
    P[2] = z;
}

/* ------------------------------------------------------------------------ */
/* sensitivity probe (not part of the method)                                */

/* SplitMix64 finaliser (Steele, Lea, Flood 2014): a counter-based generator,
 * so a noise value depends only on its key (pixel, iteration, entry, seed). */
static unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    return x ^ (x >> 31);
}

/* uniform in [-1, 1) */
static double noise_at(unsigned long long key) {
    return (double)(splitmix64(key) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* The probe adds noise a x |scale| to chosen intermediate values, x uniform
 * in [-1, 1) keyed by (pixel, iteration, entry, seed).  The scale of each
 * entry is the bound that summation in floating point obeys (the rounding of
 * a sum of terms t_i is at most a multiple of u sum |t_i|), with sum |t_i|
 * bounded by Cauchy-Schwarz in terms of the diagonal: for the normal matrix
 * N = J^T W J, sum |w j_a j_c| <= sqrt(N_aa N_cc); for the right-hand side
 * sum |w eps j_a| <= sqrt(N_aa E), E = sum w eps^2; likewise for the sums M
 * and v of the initial-normal regression (v with the sum of squared centred
 * heights).  So entry (a, c) moves by up to a sqrt(N_aa N_cc): relative to
 * the Jacobi-scaled matrix D N D, D = diag(N)^-1/2, that the solve factorises,
 * every entry moves by up to a (a = perturb).  Each coordinate of p' (and of
 * the regression's patch points relative to the centre pixel's point) is
 * multiplied by 1 + a' x (a' = perturb_points).  The method's output under
 * this noise tells how far rounding of that size can move it: the tests use
 * it to find the pixels whose answer is fixed at single precision. */
static void perturb_system(const or_params* p, unsigned long long key, double N[36], double rhs[6],
                           double E) {
    if (!(p->perturb > 0.0)) return;
    double d[6];
    for (int a = 0; a < 6; a++) d[a] = sqrt(fabs(N[7 * a]));
    for (int a = 0; a < 6; a++) {
        for (int c = a; c < 6; c++) {
            const double e = p->perturb * noise_at(key * 64 + (unsigned long long)(6 * a + c)) * d[a] * d[c];
            N[6 * a + c] += e;
            if (c != a) N[6 * c + a] += e;
        }
        rhs[a] += p->perturb * noise_at(key * 64 + 36 + (unsigned long long)a) * d[a] * sqrt(fabs(E));
    }
}

/* ------------------------------------------------------------------------ */
/* step 2: initial normal (Sec. 3.2.1, Eq. initialnormal)                   */

static int initial_normal_keyed(const double* depth, int H, int W, const or_params* p, int u0,
                                int v0, double n[3], unsigned long long key);

/* Calibration of the probe (not the method): the centred sums M and v of the
 * regression below as single-precision arithmetic forms them, in the same two
 * passes (means, then centred products) over points whose coordinates are
 * taken relative to the centre pixel's point and rounded to single
 * precision, every term and every running sum rounded to single precision. */
static void regression_sums_f32(const double* depth, int H, int W, const or_params* p, int u0, int v0,
                                double* m00, double* m01, double* m11, double* v0s, double* v1s) {
    const int rn = p->rn;
    double P0[3], P[3];
    or_backproject(p, u0, v0, depth[(size_t)v0 * W + u0], P0);
    float q[3], sq[3] = {0.0f, 0.0f, 0.0f}, acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    int cnt = 0;
    for (int pass = 0; pass < 2; pass++) {
        const float mean[3] = {sq[0] / (float)(cnt > 0 ? cnt : 1), sq[1] / (float)(cnt > 0 ? cnt : 1),
                               sq[2] / (float)(cnt > 0 ? cnt : 1)};
        for (int v = v0 - rn; v <= v0 + rn; v++)
            for (int u = u0 - rn; u <= u0 + rn; u++) {
                if (u < 0 || v < 0 || u >= W || v >= H) continue;
                const double z = depth[(size_t)v * W + u];
                if (!range_valid(z)) continue;
                or_backproject(p, u, v, z, P);
                for (int c = 0; c < 3; c++) q[c] = (float)(P[c] - P0[c]);
                if (pass == 0) {
                    for (int c = 0; c < 3; c++) sq[c] = sq[c] + q[c];
                    cnt++;
                } else {
                    const float dx = q[0] - mean[0], dy = q[1] - mean[1], dz = q[2] - mean[2];
                    const float t[5] = {dx * dx, dx * dy, dy * dy, dx * dz, dy * dz};
                    for (int c = 0; c < 5; c++) acc[c] = acc[c] + t[c];
                }
            }
    }
    *m00 = acc[0]; *m01 = acc[1]; *m11 = acc[2]; *v0s = acc[3]; *v1s = acc[4];
}

OR_EXPORT int or_initial_normal(const double* depth, int H, int W, const or_params* p, int u0,
                                int v0, double n[3]) {
    return initial_normal_keyed(depth, H, W, p, u0, v0, n, p->perturb_seed);
}

/* The centred sums of the regression over the valid points of the
 * (2 rn + 1)^2 patch around (u0, v0):
 *   sums = (M00, M01, M11, v0, v1, S_zz), M = sum (x-mx, y-my)(x-mx, y-my)^T,
 *   v = sum (x-mx, y-my)(z-mz), S_zz = sum (z-mz)^2 (the probe's scale of v);
 * single precision when p->f32_sums.  Returns the count of valid points (the
 * sums are left 0 below 3). */
/* The probe's noise on a patch point: its coordinates relative to the centre
 * pixel's point P0 multiplied by 1 + a' x (a' = perturb_points), as for p' in
 * the fitting window; keyed by the point's place in the patch. */
static void perturb_patch_point(const or_params* p, unsigned long long key, int slot, const double P0[3],
                                double P[3]) {
    if (!(p->perturb_points > 0.0)) return;
    for (int c = 0; c < 3; c++)
        P[c] = P0[c] + (P[c] - P0[c]) *
                           (1.0 + p->perturb_points * noise_at((key + 700) * 4096 + (unsigned long long)(3 * slot + c)));
}

static int regression_sums(const double* depth, int H, int W, const or_params* p, int u0, int v0,
                           double sums[6], unsigned long long key) {
    const int rn = p->rn, side = 2 * rn + 1;
    double P[3], P0[3], sx = 0.0, sy = 0.0, sz = 0.0;
    or_backproject(p, u0, v0, depth[(size_t)v0 * W + u0], P0);
    int cnt = 0;
    for (int i = 0; i < 6; i++) sums[i] = 0.0;
    for (int v = v0 - rn; v <= v0 + rn; v++)
        for (int u = u0 - rn; u <= u0 + rn; u++) {
            if (u < 0 || v < 0 || u >= W || v >= H) continue;
            double z = depth[(size_t)v * W + u];
            if (!range_valid(z)) continue;
            or_backproject(p, u, v, z, P);
            perturb_patch_point(p, key, (v - v0 + rn) * side + (u - u0 + rn), P0, P);
            sx += P[0]; sy += P[1]; sz += P[2];
            cnt++;
        }
    if (cnt < 3) return cnt;
    const double mx = sx / cnt, my = sy / cnt, mz = sz / cnt;
    double m00 = 0.0, m01 = 0.0, m11 = 0.0, v0s = 0.0, v1s = 0.0, szz = 0.0;
    for (int v = v0 - rn; v <= v0 + rn; v++)
        for (int u = u0 - rn; u <= u0 + rn; u++) {
            if (u < 0 || v < 0 || u >= W || v >= H) continue;
            double z = depth[(size_t)v * W + u];
            if (!range_valid(z)) continue;
            or_backproject(p, u, v, z, P);
            perturb_patch_point(p, key, (v - v0 + rn) * side + (u - u0 + rn), P0, P);
            const double dx = P[0] - mx, dy = P[1] - my, dz = P[2] - mz;
            m00 += dx * dx; m01 += dx * dy; m11 += dy * dy;
            v0s += dx * dz; v1s += dy * dz;
            szz += dz * dz;
        }
    if (p->f32_sums) regression_sums_f32(depth, H, W, p, u0, v0, &m00, &m01, &m11, &v0s, &v1s);
    sums[0] = m00; sums[1] = m01; sums[2] = m11; sums[3] = v0s; sums[4] = v1s; sums[5] = szz;
    return cnt;
}

OR_EXPORT int or_regression_sums(const double* depth, int H, int W, const or_params* p, int u0, int v0,
                                 double sums[6]) {
    or_params q = *p;
    q.perturb_points = 0.0;
    return regression_sums(depth, H, W, &q, u0, v0, sums, 0);
}

static int initial_normal_keyed(const double* depth, int H, int W, const or_params* p, int u0,
                                int v0, double n[3], unsigned long long key) {
    double S[6];
    if (regression_sums(depth, H, W, p, u0, v0, S, key) < 3) return OR_BAD_NORMAL;
    double m00 = S[0], m01 = S[1], m11 = S[2], v0s = S[3], v1s = S[4];
    if (p->perturb > 0.0) { /* the probe, scaled as for the normal equations */
        const double d0 = sqrt(fabs(m00)), d1 = sqrt(fabs(m11)), dz = sqrt(fabs(S[5]));
        m00 += p->perturb * noise_at(key * 64 + 50) * d0 * d0;
        m01 += p->perturb * noise_at(key * 64 + 51) * d0 * d1;
        m11 += p->perturb * noise_at(key * 64 + 52) * d1 * d1;
        v0s += p->perturb * noise_at(key * 64 + 53) * d0 * dz;
        v1s += p->perturb * noise_at(key * 64 + 54) * d1 * dz;
    }
    const double det = m00 * m11 - m01 * m01, tr = m00 + m11;
    if (!(det > p->det_tol * tr * tr)) return OR_BAD_NORMAL;
    /* (a, b)^T = M^-1 v by the 2x2 inverse */
    const double a = (m11 * v0s - m01 * v1s) / det;
    const double b = (m00 * v1s - m01 * v0s) / det;
    const double s = 1.0 / sqrt(1.0 + a * a + b * b);
    n[0] = -a * s; n[1] = -b * s; n[2] = s;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* step 3: frame whose local z axis is the normal (Sec. 3.2.2)              */

/* The minimal rotation with R n = e_z (Rodrigues' formula for the rotation
 * taking unit n to unit e_z: w = n x e_z, c = n . e_z,
 * R = I + [w]_x + [w]_x^2 / (1 + c)).  Requires n_z > -1. */
OR_EXPORT void or_frame_from_normal(const double n[3], double R[9]) {
    const double w[3] = {n[1], -n[0], 0.0};
    const double c = n[2];
    double S[9], S2[9];
    skew(w, S);
    mat3_mul(S, S, S2);
    for (int i = 0; i < 9; i++) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + S[i] + S2[i] / (1.0 + c);
}

/* rotation by angle |w| about axis w/|w| (exponential map), Rodrigues */
OR_EXPORT void or_rotation_exp(const double w[3], double R[9]) {
    const double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int i = 0; i < 9; i++) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    if (th == 0.0) return;
    const double ax[3] = {w[0] / th, w[1] / th, w[2] / th};
    double K[9], K2[9];
    skew(ax, K);
    mat3_mul(K, K, K2);
    const double s = sin(th), c1 = 1.0 - cos(th);
    for (int i = 0; i < 9; i++) R[i] += s * K[i] + c1 * K2[i];
}

/* ------------------------------------------------------------------------ */
/* step 4: E, Q and the residual (Sec. 3.1.2, Eq. quad; Eq. error_func)      */

/* E = [[R, (0,0,tz)^T], [0 0 0 1]] */
static void make_E(const double R[9], double tz, double E[16]) {
    memset(E, 0, 16 * sizeof(double));
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) E[4 * i + j] = R[3 * i + j];
    E[4 * 2 + 3] = tz;
    E[15] = 1.0;
}

/* Q of the parabolic patch z = A/2 x^2 + B x y + C/2 y^2 */
static void make_Q(double A, double B, double C, double Q[16]) {
    memset(Q, 0, 16 * sizeof(double));
    Q[0] = A / 2.0;  Q[1] = B / 2.0;
    Q[4] = B / 2.0;  Q[5] = C / 2.0;
    Q[4 * 2 + 3] = -0.5;
    Q[4 * 3 + 2] = -0.5;
}

/* Residual eps = p~^T E^T Q E p~ of one p-relative point p' and its Jacobian
 * j = d eps / d(theta_x, theta_y, t_z, A, B, C) (Sec. 3.2.3).
 *   rotation: R -> Rot(theta) R with Rot(theta) = exp([theta]_x), so
 *             dE/dtheta_a = [[ [e_a]_x R, 0 ], [0, 0]];
 *   offset:   dE/dt_z has a single 1 at row 2, column 3;
 *   since Q is symmetric, d eps/d(param of E) = 2 (E p~)^T Q (dE p~),
 *   and d eps/d(param of Q) = (E p~)^T (dQ) (E p~). */
OR_EXPORT void or_residual(const double R[9], double tz, double A, double B, double C,
                           const double pp[3], double* eps, double j[6]) {
    double E[16], Q[16], Ep[4], QEp[4];
    const double pt[4] = {pp[0], pp[1], pp[2], 1.0};
    make_E(R, tz, E);
    make_Q(A, B, C, Q);
    mat4_vec(E, pt, Ep);
    mat4_vec(Q, Ep, QEp);
    *eps = dot4(Ep, QEp);
    if (!j) return;
    for (int a = 0; a < 2; a++) {
        double e[3] = {0.0, 0.0, 0.0}, S[9], SR[9], dE[16], dEp[4];
        e[a] = 1.0;
        skew(e, S);
        mat3_mul(S, R, SR);
        memset(dE, 0, sizeof dE);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) dE[4 * r + c] = SR[3 * r + c];
        mat4_vec(dE, pt, dEp);
        j[a] = 2.0 * dot4(QEp, dEp);
    }
    {
        double dE[16], dEp[4];
        memset(dE, 0, sizeof dE);
        dE[4 * 2 + 3] = 1.0;
        mat4_vec(dE, pt, dEp);
        j[2] = 2.0 * dot4(QEp, dEp);
    }
    for (int q = 0; q < 3; q++) {
        double dQ[16], dQEp[4];
        memset(dQ, 0, sizeof dQ);
        if (q == 0) dQ[0] = 0.5;
        if (q == 1) { dQ[1] = 0.5; dQ[4] = 0.5; }
        if (q == 2) dQ[5] = 0.5;
        mat4_vec(dQ, Ep, dQEp);
        j[3 + q] = dot4(Ep, dQEp);
    }
}

/* ------------------------------------------------------------------------ */
/* steps 6-7: one re-weighted update (Sec. 3.2.3)                            */

/* Weighting function W(eps) = k / (k + eps^2); with rejection it is 0 unless
 * eps^2 <= R, R = reject_ratio * mse (Eq. weighting_function). */
OR_EXPORT double or_weight(const or_params* p, double eps, double mse) {
    const double e2 = eps * eps;
    if (p->reject && !(e2 <= p->reject_ratio * mse)) return 0.0;
    return p->k / (p->k + e2);
}

/* Solve N b = rhs for symmetric positive definite N (6x6) by Cholesky of the
 * Jacobi-scaled matrix S = D N D, D = diag(N)^-1/2 (same solution; the scaled
 * pivots decide singularity).  Returns 0, or OR_SINGULAR.  *cond becomes at
 * least the ratio of the largest to the smallest pivot seen (infinite when a
 * pivot is not positive). */
static int solve6(const double N[36], const double rhs[6], double tol, double b[6],
                  double* min_pivot, double* cond) {
    double D[6], S[36], L[36], y[6], z[6];
    for (int i = 0; i < 6; i++) {
        if (!(N[7 * i] > 0.0)) {
            *cond = INFINITY;
            return OR_SINGULAR;
        }
        D[i] = 1.0 / sqrt(N[7 * i]);
    }
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < 6; j++) S[6 * i + j] = D[i] * N[6 * i + j] * D[j];
    memset(L, 0, sizeof L);
    double pmax = 0.0;
    for (int j = 0; j < 6; j++) {
        double piv = S[7 * j];
        for (int k = 0; k < j; k++) piv -= L[6 * j + k] * L[6 * j + k];
        if (piv < *min_pivot) *min_pivot = piv;
        if (piv > pmax) pmax = piv;
        const double ratio = piv > 0.0 ? pmax / piv : INFINITY;
        if (!(ratio <= *cond)) *cond = ratio;
        if (!(piv > tol)) return OR_SINGULAR;
        L[7 * j] = sqrt(piv);
        for (int i = j + 1; i < 6; i++) {
            double s = S[6 * i + j];
            for (int k = 0; k < j; k++) s -= L[6 * i + k] * L[6 * j + k];
            L[6 * i + j] = s / L[7 * j];
        }
    }
    for (int i = 0; i < 6; i++) y[i] = D[i] * rhs[i];
    for (int i = 0; i < 6; i++) { /* L z = y */
        double s = y[i];
        for (int k = 0; k < i; k++) s -= L[6 * i + k] * z[k];
        z[i] = s / L[7 * i];
    }
    for (int i = 5; i >= 0; i--) { /* L^T y = z */
        double s = z[i];
        for (int k = i + 1; k < 6; k++) s -= L[6 * k + i] * y[k];
        y[i] = s / L[7 * i];
    }
    for (int i = 0; i < 6; i++) b[i] = D[i] * y[i];
    return OR_OK;
}

/* TF32 of a single-precision number (10 explicit mantissa bits, rounded to
 * nearest with ties away from zero), as tensor cores read their operands. */
static float to_tf32(float x) {
    unsigned int u;
    memcpy(&u, &x, sizeof u);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
    float y;
    memcpy(&y, &u, sizeof y);
    return y;
}

/* Calibration of the probe (not the method): the normal equations of one
 * iteration as single-precision arithmetic forms them.  Every term of every
 * sum (w j_a j_c, w eps j_a) is rounded to single precision and added to a
 * single-precision running sum in the plain order of the points.  The terms
 * themselves come from the same double-precision residuals, Jacobian and
 * weights as the method's own loop, so the result differs from it by the
 * rounding of the sums alone (and of p', which the caller rounds).
 * f32_sums = 2 or 3 forms the terms of J^T W J as tensor cores would from
 * the single-precision features f_a = sqrt(w) j_a: 2 = one product of their
 * TF32 parts, 3 = TF32 parts split in two, hi hi + hi lo + lo hi. */
static void normal_equations_f32(const or_params* p, const double* eps, const double* J, int m,
                                 double mse, double N[36], double rhs[6], double* w_out) {
    float n32[36], r32[6];
    for (int a = 0; a < 36; a++) n32[a] = 0.0f;
    for (int a = 0; a < 6; a++) r32[a] = 0.0f;
    for (int i = 0; i < m; i++) {
        const double wi = or_weight(p, eps[i], mse);
        if (w_out) w_out[i] = wi;
        const double* row = J + 6 * i;
        float hi[6], lo[6];
        for (int a = 0; a < 6; a++) {
            const float f = (float)(sqrt(wi) * row[a]);
            hi[a] = to_tf32(f);
            lo[a] = to_tf32(f - hi[a]);
        }
        for (int a = 0; a < 6; a++) {
            for (int c = 0; c < 6; c++) {
                const float term = p->f32_sums == 2   ? hi[a] * hi[c]
                                   : p->f32_sums == 3 ? hi[a] * hi[c] + (hi[a] * lo[c] + lo[a] * hi[c])
                                                      : (float)(row[a] * wi * row[c]);
                n32[6 * a + c] = n32[6 * a + c] + term;
            }
            const float term = (float)(row[a] * wi * eps[i]);
            r32[a] = r32[a] + term;
        }
    }
    for (int a = 0; a < 36; a++) N[a] = (double)n32[a];
    for (int a = 0; a < 6; a++) rhs[a] = (double)r32[a];
}

/* One iteration over the m p-relative points pts (m x 3): residuals and
 * Jacobian at the current state, weights, the normal equations
 * N = J^T W J, rhs = J^T W eps, b = N^-1 rhs, and the update
 * (theta_x, theta_y, t_z, A, B, C) <- (...) - b, the rotation part applied as
 * R <- Rot(-b_0, -b_1, 0) R.  Optional outputs N (36), rhs (6), b (6) and the
 * weights (m).  Returns OR_OK or OR_SINGULAR (state then unchanged). */
static int irls_step_keyed(const double* pts, int m, const or_params* p, double R[9], double* tz,
                           double* A, double* B, double* C, double* min_pivot, double* cond,
                           double* N_out, double* rhs_out, double* b_out, double* w_out,
                           unsigned long long key);

OR_EXPORT int or_irls_step(const double* pts, int m, const or_params* p, double R[9], double* tz,
                           double* A, double* B, double* C, double* min_pivot, double* N_out,
                           double* rhs_out, double* b_out, double* w_out) {
    return irls_step_keyed(pts, m, p, R, tz, A, B, C, min_pivot, NULL, N_out, rhs_out, b_out, w_out,
                           p->perturb_seed);
}

static int irls_step_keyed(const double* pts, int m, const or_params* p, double R[9], double* tz,
                           double* A, double* B, double* C, double* min_pivot, double* cond,
                           double* N_out, double* rhs_out, double* b_out, double* w_out,
                           unsigned long long key) {
    double N[36], rhs[6], b[6], mp = 1.0, cd = 1.0;
    double* eps = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double* J = (double*)malloc(sizeof(double) * 6 * (size_t)(m > 0 ? m : 1));
    double mse = 0.0;
    for (int i = 0; i < m; i++) {
        or_residual(R, *tz, *A, *B, *C, pts + 3 * i, &eps[i], J + 6 * i);
        mse += eps[i] * eps[i];
    }
    mse = m > 0 ? mse / m : 0.0;
    memset(N, 0, sizeof N);
    memset(rhs, 0, sizeof rhs);
    if (p->f32_sums) {
        normal_equations_f32(p, eps, J, m, mse, N, rhs, w_out);
    } else {
        for (int i = 0; i < m; i++) {
            const double w = or_weight(p, eps[i], mse);
            if (w_out) w_out[i] = w;
            const double* ji = J + 6 * i;
            for (int a = 0; a < 6; a++) {
                for (int c = 0; c < 6; c++) N[6 * a + c] += ji[a] * w * ji[c];
                rhs[a] += ji[a] * w * eps[i];
            }
        }
    }
    double E = 0.0; /* sum w eps^2, the probe's scale of the right-hand side */
    if (p->perturb > 0.0)
        for (int i = 0; i < m; i++) E += or_weight(p, eps[i], mse) * eps[i] * eps[i];
    free(eps);
    free(J);
    perturb_system(p, key, N, rhs, E);
    if (N_out) memcpy(N_out, N, sizeof N);
    if (rhs_out) memcpy(rhs_out, rhs, sizeof rhs);
    const int st = solve6(N, rhs, p->pivot_tol, b, &mp, &cd);
    if (min_pivot && mp < *min_pivot) *min_pivot = mp;
    if (cond && !(cd <= *cond)) *cond = cd;
    if (st != OR_OK) return st;
    if (b_out) memcpy(b_out, b, sizeof b);
    const double w[3] = {-b[0], -b[1], 0.0};
    double Rd[9], Rn[9];
    or_rotation_exp(w, Rd);
    mat3_mul(Rd, R, Rn);
    memcpy(R, Rn, sizeof Rn);
    *tz -= b[2];
    *A -= b[3];
    *B -= b[4];
    *C -= b[5];
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* step 8: principal curvatures (Sec. 3.1.2)                                */

/* T1 = (A + C)/2, T2 = sqrt(T1^2 - AC + B^2), k1 = T1 + T2, k2 = T1 - T2.
 * T1^2 - AC + B^2 is evaluated as ((A - C)/2)^2 + B^2, the same number in
 * exact arithmetic, which cannot turn negative by rounding. */
OR_EXPORT void or_principal(double A, double B, double C, double* k1, double* k2) {
    const double T1 = (A + C) / 2.0;
    const double h = (A - C) / 2.0;
    const double T2 = sqrt(h * h + B * B);
    *k1 = T1 + T2;
    *k2 = T1 - T2;
}

/* ------------------------------------------------------------------------ */
/* the window and the whole per-pixel method                                 */

/* Lists the valid pixels of the (2r+1)^2 window around (u0, v0) sampled on the
 * stride (offsets that are multiples of stride, |offset| <= r), clipped to the
 * image, centre included.  Writes up to max (u, v) pairs; returns the count. */
OR_EXPORT int or_window(const double* depth, int H, int W, const or_params* p, int u0, int v0,
                        int* uv, int max) {
    const int r = p->r, s = p->stride > 0 ? p->stride : 1;
    int cnt = 0;
    for (int dv = -(r / s) * s; dv <= r; dv += s)
        for (int du = -(r / s) * s; du <= r; du += s) {
            const int u = u0 + du, v = v0 + dv;
            if (u < 0 || v < 0 || u >= W || v >= H) continue;
            if (!range_valid(depth[(size_t)v * W + u])) continue;
            if (uv && cnt < max) {
                uv[2 * cnt] = u;
                uv[2 * cnt + 1] = v;
            }
            cnt++;
        }
    return cnt;
}

static void fail(or_result* res, int status) {
    const double nan = NAN;
    res->status = status;
    res->k1 = res->k2 = nan;
    res->normal[0] = res->normal[1] = res->normal[2] = nan;
}

OR_EXPORT int or_fit_pixel(const double* depth, int H, int W, const or_params* p, int u0, int v0,
                           or_result* res) {
    memset(res, 0, sizeof *res);
    res->min_pivot = 1.0;
    res->cond = 1.0;
    const double z0 = depth[(size_t)v0 * W + u0];
    if (!range_valid(z0)) { fail(res, OR_INVALID_CENTRE); return res->status; }
    const unsigned long long pkey =
        splitmix64(p->perturb_seed ^ splitmix64(((unsigned long long)v0 << 32) ^ (unsigned long long)u0));
    double n[3];
    if (initial_normal_keyed(depth, H, W, p, u0, v0, n, pkey * 1024) != OR_OK) {
        fail(res, OR_BAD_NORMAL);
        return res->status;
    }
    memcpy(res->n0, n, sizeof n);
    double R[9], tz = 0.0, A = 0.0, B = 0.0, C = 0.0;
    or_frame_from_normal(n, R);

    const int side = 2 * p->r + 1;
    int* uv = (int*)malloc(sizeof(int) * 2 * (size_t)side * side);
    const int m = or_window(depth, H, W, p, u0, v0, uv, side * side);
    res->npts = m;
    if (m < p->min_window) { free(uv); fail(res, OR_FEW_POINTS); return res->status; }
    /* p'_i = p_i - p (Sec. 3.1.2) */
    double P0[3], Pi[3];
    or_backproject(p, u0, v0, z0, P0);
    double* pts = (double*)malloc(sizeof(double) * 3 * (size_t)m);
    for (int i = 0; i < m; i++) {
        const int u = uv[2 * i], v = uv[2 * i + 1];
        or_backproject(p, u, v, depth[(size_t)v * W + u], Pi);
        for (int c = 0; c < 3; c++) pts[3 * i + c] = Pi[c] - P0[c];
        if (p->perturb_points > 0.0)
            for (int c = 0; c < 3; c++)
                pts[3 * i + c] *= 1.0 + p->perturb_points *
                                           noise_at((pkey * 1024 + 512) * 4096 + (unsigned long long)(3 * i + c));
        if (p->f32_sums)  /* calibration: p' as a single-precision number */
            for (int c = 0; c < 3; c++) pts[3 * i + c] = (double)(float)pts[3 * i + c];
    }
    free(uv);
    double mp = 1.0, cd = 1.0;
    for (int t = 0; t < p->T; t++) {
        const unsigned long long key = pkey * 1024 + 1 + (unsigned long long)t;
        if (irls_step_keyed(pts, m, p, R, &tz, &A, &B, &C, &mp, &cd, NULL, NULL, res->last_b, NULL, key) !=
            OR_OK) {
            free(pts);
            res->min_pivot = mp;
            res->cond = cd;
            res->iters = t;
            fail(res, OR_SINGULAR);
            return res->status;
        }
        res->iters = t + 1;
    }
    free(pts);
    res->min_pivot = mp;
    res->cond = cd;
    res->A = A; res->B = B; res->C = C; res->tz = tz;
    memcpy(res->R, R, sizeof R);
    or_principal(A, B, C, &res->k1, &res->k2);
    /* refined normal: the local z axis in camera coordinates, R^T e_z (Sec. 3.2.4) */
    res->normal[0] = R[6]; res->normal[1] = R[7]; res->normal[2] = R[8];
    res->status = OR_OK;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* whole images                                                              */

static void store(const or_result* r, size_t i, double* k1, double* k2, double* normal,
                  int* status, double* min_pivot, double* last_b, double* cond) {
    if (cond) cond[i] = r->cond;
    if (last_b) for (int c = 0; c < 6; c++) last_b[6 * i + c] = r->last_b[c];
    if (k1) k1[i] = r->k1;
    if (k2) k2[i] = r->k2;
    if (normal) for (int c = 0; c < 3; c++) normal[3 * i + c] = r->normal[c];
    if (status) status[i] = r->status;
    if (min_pivot) min_pivot[i] = r->min_pivot;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* threads the library would use for a parallel loop (1 without OpenMP) */
OR_EXPORT int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* All pixels of a double-precision range image; outputs are H*W (normal
 * H*W*3, last_b H*W*6, cond H*W), any of them may be NULL.  Pixels are independent;
 * nthreads > 0 sets the OpenMP thread count. */
OR_EXPORT void or_curvature_image_f64(const double* depth, int H, int W, const or_params* p,
                                      double* k1, double* k2, double* normal, int* status,
                                      double* min_pivot, double* last_b, double* cond, int nthreads) {
    set_threads(nthreads);
    const long npx = (long)H * W;
#pragma omp parallel for schedule(dynamic, 8)
    for (long i = 0; i < npx; i++) {
        or_result r;
        or_fit_pixel(depth, H, W, p, (int)(i % W), (int)(i / W), &r);
        store(&r, (size_t)i, k1, k2, normal, status, min_pivot, last_b, cond);
    }
}

/* The same for the n pixels listed in uv (n x 2, (u, v)); outputs are n long. */
OR_EXPORT void or_curvature_pixels_f64(const double* depth, int H, int W, const or_params* p,
                                       const int* uv, int n, double* k1, double* k2,
                                       double* normal, int* status, double* min_pivot,
                                       double* last_b, double* cond, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 8)
    for (int i = 0; i < n; i++) {
        or_result r;
        or_fit_pixel(depth, H, W, p, uv[2 * i], uv[2 * i + 1], &r);
        store(&r, (size_t)i, k1, k2, normal, status, min_pivot, last_b, cond);
    }
}

/* float32 range images are widened exactly to double first */
static double* widen(const float* d, long npx) {
    double* o = (double*)malloc(sizeof(double) * (size_t)(npx > 0 ? npx : 1));
    for (long i = 0; i < npx; i++) o[i] = (double)d[i];
    return o;
}

OR_EXPORT void or_curvature_image(const float* depth, int H, int W, const or_params* p, double* k1,
                                  double* k2, double* normal, int* status, double* min_pivot,
                                  double* last_b, double* cond, int nthreads) {
    double* d = widen(depth, (long)H * W);
    or_curvature_image_f64(d, H, W, p, k1, k2, normal, status, min_pivot, last_b, cond, nthreads);
    free(d);
}

OR_EXPORT void or_curvature_pixels(const float* depth, int H, int W, const or_params* p,
                                   const int* uv, int n, double* k1, double* k2, double* normal,
                                   int* status, double* min_pivot, double* last_b, double* cond, int nthreads) {
    double* d = widen(depth, (long)H * W);
    or_curvature_pixels_f64(d, H, W, p, uv, n, k1, k2, normal, status, min_pivot, last_b, cond, nthreads);
    free(d);
}

OR_EXPORT int or_fit_pixel_f32(const float* depth, int H, int W, const or_params* p, int u0, int v0,
                               or_result* res) {
    double* d = widen(depth, (long)H * W);
    const int st = or_fit_pixel(d, H, W, p, u0, v0, res);
    free(d);
    return st;
}

/* ------------------------------------------------------------------------ */
/* organised outputs: the back-projection and the initial normals of every   */
/* pixel on their own (Sec. 3, Sec. 3.2.1), for the point-cloud and          */
/* normal-field outputs                                                      */

/* xyz: H*W*3, NaN where the range is not valid */
OR_EXPORT void or_backproject_image(const float* depth, int H, int W, const or_params* p, double* xyz) {
    const long npx = (long)H * W;
    for (long i = 0; i < npx; i++) {
        const double z = (double)depth[i];
        if (!range_valid(z)) {
            xyz[3 * i] = xyz[3 * i + 1] = xyz[3 * i + 2] = NAN;
            continue;
        }
        or_backproject(p, (int)(i % W), (int)(i / W), z, xyz + 3 * i);
    }
}

/* normal: H*W*3 (NaN unless status is OR_OK); status: H*W, OR_INVALID_CENTRE
 * for an invalid range, OR_BAD_NORMAL when the regression fails.  With
 * p->perturb > 0 the regression sums are perturbed under the same per-pixel
 * keys as in or_fit_pixel. */
OR_EXPORT void or_initial_normal_image(const float* depth, int H, int W, const or_params* p, double* normal,
                                       int* status, int nthreads) {
    set_threads(nthreads);
    const long npx = (long)H * W;
    double* d = widen(depth, npx);
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < npx; i++) {
        const int u0 = (int)(i % W), v0 = (int)(i / W);
        double* n = normal + 3 * i;
        n[0] = n[1] = n[2] = NAN;
        if (!range_valid(d[i])) {
            status[i] = OR_INVALID_CENTRE;
            continue;
        }
        const unsigned long long pkey =
            splitmix64(p->perturb_seed ^ splitmix64(((unsigned long long)v0 << 32) ^ (unsigned long long)u0));
        double m[3];
        status[i] = initial_normal_keyed(d, H, W, p, u0, v0, m, pkey * 1024);
        if (status[i] == OR_OK) memcpy(n, m, sizeof m);
    }
    free(d);
}
