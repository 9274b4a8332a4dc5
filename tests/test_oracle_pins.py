"""Pins of the FP64 oracle against things other than itself: closed forms,
finite differences, library least squares and eigenvalues, brute force, and
invariants of the method (Spek, Li, Drummond, arXiv 1707.00385, Sec. 3).

Every check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or index, a transposed operand) fails at least one of them."""
import itertools

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], dtype=float)


def rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = skew(axis)
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


# ---------------------------------------------------------------- step 1

def test_backproject_reprojects(orc):
    """Sec. 3.2 input: P projects back to its pixel through the pinhole model."""
    p = orc.params(525.0, 530.0, 319.5, 239.5, r=7, T=5)
    for (u, v, z) in [(0, 0, 1.0), (639, 479, 3.25), (100, 400, 0.5), (320, 240, 2.0)]:
        P = orc.backproject(p, u, v, z)
        assert P[2] == z
        assert abs(525.0 * P[0] / P[2] + 319.5 - u) < 1e-9
        assert abs(530.0 * P[1] / P[2] + 239.5 - v) < 1e-9


# ---------------------------------------------------------------- step 2

def plane_depth(cam, n, d):
    t, _, _, _ = synth.Plane(np.asarray(n, float) / np.linalg.norm(n), d).hit(cam.rays())
    return np.where(np.isfinite(t), t, 0.0)


@pytest.mark.parametrize("n", [(0, 0, 1), (0.3, -0.2, 1), (-0.6, 0.1, 1), (0.1, 0.8, 1)])
def test_initial_normal_of_plane(orc, n):
    """Sec. 3.2.1: on noise-free points of a plane the regression z = a x + b y + c
    is exact, so Eq. initialnormal gives the plane normal."""
    cam = synth.Camera(40, 50, 60.0, 62.0, 24.5, 19.5)
    n = np.asarray(n, float) / np.linalg.norm(n)
    depth = plane_depth(cam, n, 1.3)
    p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=3, T=1)
    for (u, v) in [(25, 20), (3, 3), (0, 0), (49, 39)]:
        st, n0 = orc.initial_normal(depth, p, u, v)
        assert st == orc.OK
        assert np.allclose(n0, n if n[2] > 0 else -n, atol=1e-10)


def test_initial_normal_vs_lstsq(orc):
    """Sec. 3.2.1 on noisy points with holes: (a, b) equal the slopes of a
    library least-squares fit of z on (1, x, y) over the same valid points."""
    rng = np.random.default_rng(3)
    cam = synth.Camera(30, 30, 40.0, 40.0, 14.0, 15.0)
    depth = 1.5 + 0.05 * rng.standard_normal((30, 30))
    depth[rng.random((30, 30)) < 0.2] = 0.0
    p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=3, T=1)
    for (u, v) in [(10, 12), (0, 29), (15, 15), (29, 1)]:
        if depth[v, u] == 0:
            continue
        pts = []
        for vv in range(v - 3, v + 4):
            for uu in range(u - 3, u + 4):
                if 0 <= uu < 30 and 0 <= vv < 30 and depth[vv, uu] > 0:
                    pts.append(orc.backproject(p, uu, vv, depth[vv, uu]))
        pts = np.array(pts)
        X = np.c_[np.ones(len(pts)), pts[:, 0], pts[:, 1]]
        coef = np.linalg.lstsq(X, pts[:, 2], rcond=None)[0]
        a, b = coef[1], coef[2]
        st, n0 = orc.initial_normal(depth, p, u, v)
        assert st == orc.OK
        ref = np.array([-a, -b, 1.0]) / np.sqrt(1 + a * a + b * b)
        assert np.allclose(n0, ref, atol=1e-10)


def test_initial_normal_degenerate(orc):
    """Fewer than 3 points, or all points on one image row (collinear in x, y),
    leave the regression undetermined."""
    p = orc.params(50.0, 50.0, 10.0, 10.0, r=2, T=1)
    d = np.zeros((20, 20))
    d[10, 10] = d[10, 11] = 1.0
    assert orc.initial_normal(d, p, 10, 10)[0] == orc.BAD_NORMAL
    d[10, 5:16] = 1.0 + 0.01 * np.arange(11)   # one row: (X, Y) collinear
    assert orc.initial_normal(d, p, 10, 10)[0] == orc.BAD_NORMAL
    d[11, 9] = 1.0
    assert orc.initial_normal(d, p, 10, 10)[0] == orc.OK


# ---------------------------------------------------------------- step 3

@pytest.mark.parametrize("n", [(0, 0, 1), (0.2, 0.1, 1), (-0.9, 0.4, 0.3), (0.01, -0.02, 1)])
def test_frame_from_normal(orc, n):
    """Sec. 3.2.2: R maps the normal to the local z axis, is a proper rotation,
    and is the smallest such rotation (angle acos n_z about an axis in the
    x-y plane, i.e. no spin about z)."""
    n = np.asarray(n, float) / np.linalg.norm(n)
    R = orc.frame_from_normal(n)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert abs(np.linalg.det(R) - 1) < 1e-14
    assert np.allclose(R @ n, [0, 0, 1], atol=1e-14)
    ang = np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1))
    assert abs(ang - np.arccos(n[2])) < 1e-7
    if ang > 1e-6:
        axis = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
        assert abs(axis[2]) < 1e-12


def test_rotation_exp_vs_expm(orc):
    from scipy.linalg import expm
    rng = np.random.default_rng(0)
    for _ in range(10):
        w = rng.normal(size=3) * rng.uniform(1e-6, 2.0)
        assert np.allclose(orc.rotation_exp(w), expm(skew(w)), atol=1e-13)
    assert np.array_equal(orc.rotation_exp(np.zeros(3)), np.eye(3))


# ---------------------------------------------------------------- step 4

def test_residual_is_parabolic_patch_equation(orc):
    """Sec. 3.1.2: at R = I, t_z = 0 the residual of (x, y, z) is
    A/2 x^2 + B x y + C/2 y^2 - z (Eq. parabolic moved to one side)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        A, B, C = rng.normal(size=3) * 10
        x, y, z = rng.normal(size=3) * 0.05
        e, _ = orc.residual(np.eye(3), 0.0, A, B, C, [x, y, z])
        assert abs(e - (A / 2 * x * x + B * x * y + C / 2 * y * y - z)) < 1e-15


def test_points_on_posed_patch_have_zero_residual(orc):
    """Eq. quad: points of the posed patch {p' : E p' on the parabola} satisfy
    p'^T E^T Q E p' = 0 for any rotation and offset (t_z after R)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        R = rot(rng.normal(size=3), rng.uniform(0, 1.2))
        tz = rng.normal() * 0.01
        A, B, C = rng.normal(size=3) * 20
        x, y = rng.normal(size=2) * 0.05
        local = np.array([x, y, A / 2 * x * x + B * x * y + C / 2 * y * y - tz])
        pp = R.T @ local
        e, _ = orc.residual(R, tz, A, B, C, pp)
        assert abs(e) < 1e-15
        # moving the point along the local z axis by d changes the residual by -d
        e2, _ = orc.residual(R, tz, A, B, C, pp + R.T @ np.array([0, 0, 1e-3]))
        assert abs(e2 + 1e-3) < 1e-15


# ---------------------------------------------------------------- step 5

def test_jacobian_by_central_differences(orc):
    """Sec. 3.2.3: j = d eps / d(theta_x, theta_y, t_z, A, B, C), the rotation
    perturbed on the left, R -> exp([theta]_x) R."""
    from scipy.linalg import expm
    rng = np.random.default_rng(4)
    for _ in range(25):
        R = rot(rng.normal(size=3), rng.uniform(0, 1.0))
        st = np.r_[rng.normal() * 0.01, rng.normal(size=3) * 15]
        pp = rng.normal(size=3) * 0.04
        _, j = orc.residual(R, *st, pp)

        def eps(delta):
            Rp = expm(skew([delta[0], delta[1], 0.0])) @ R
            e, _ = orc.residual(Rp, st[0] + delta[2], st[1] + delta[3], st[2] + delta[4], st[3] + delta[5], pp)
            return e

        h = 1e-6
        fd = np.array([(eps(h * np.eye(6)[i]) - eps(-h * np.eye(6)[i])) / (2 * h) for i in range(6)])
        assert np.allclose(j, fd, rtol=1e-6, atol=1e-9 * (1 + np.abs(fd).max()))


# ---------------------------------------------------------------- step 6

def test_weight_is_cauchy_irls_weight(orc):
    """Eq. weighting_function: W(eps) = k/(k+eps^2).  It is the IRLS weight of
    the Cauchy loss rho(e) = k/2 ln(1 + e^2/k): W(e) e = rho'(e)."""
    p = orc.params(1, 1, 0, 0, r=1, T=1, k=2.5e-4)
    k = 2.5e-4
    assert orc.weight(p, 0.0) == 1.0
    assert abs(orc.weight(p, np.sqrt(k)) - 0.5) < 1e-15
    for e in [1e-4, 3e-3, -0.02, 0.5]:
        rho = lambda t: k / 2 * np.log1p(t * t / k)
        d = 1e-7 * max(abs(e), 1e-3)
        drho = (rho(e + d) - rho(e - d)) / (2 * d)
        assert abs(orc.weight(p, e) * e - drho) < 1e-6 * abs(drho)
    es = np.linspace(0, 1, 50)
    ws = [orc.weight(p, e) for e in es]
    assert all(a > b for a, b in zip(ws, ws[1:]))


def test_weight_rejection(orc):
    """Eq. weighting_function with the rejection filter: weight 0 once
    eps^2 exceeds R = ratio * MSE; points at or below R keep k/(k+eps^2)."""
    p = orc.params(1, 1, 0, 0, r=1, T=1, k=1e-4, reject=1, reject_ratio=2.0)
    mse = 1e-4
    assert orc.weight(p, np.sqrt(2.0 * mse) * 1.001, mse) == 0.0
    e = np.sqrt(2.0 * mse) * 0.999
    assert orc.weight(p, e, mse) == pytest.approx(1e-4 / (1e-4 + e * e), rel=1e-15)
    assert orc.weight(p, 0.0, 0.0) == 1.0   # exact data keeps every point


# ---------------------------------------------------------------- step 7

def random_points(rng, m, noise=0.002, outliers=0):
    A, B, C = rng.normal(size=3) * 8
    xy = rng.uniform(-0.03, 0.03, size=(m, 2))
    z = A / 2 * xy[:, 0] ** 2 + B * xy[:, 0] * xy[:, 1] + C / 2 * xy[:, 1] ** 2 + noise * rng.standard_normal(m)
    z[:outliers] += rng.uniform(0.05, 0.2, size=outliers)
    R = rot(rng.normal(size=3), rng.uniform(0, 0.5))
    return (np.c_[xy, z] @ R), R   # p' = R^T local


@pytest.mark.parametrize("reject", [0, 1])
def test_irls_step_is_weighted_least_squares(orc, reject):
    """Eq. iter_reweighted_update: b = (J^T W J)^-1 J^T W eps equals the
    library least-squares solution of sqrt(W) J b = sqrt(W) eps, and the update
    is the Gauss-Newton step: (t_z, A, B, C) decrease by b and R turns by
    exp([-b_0, -b_1, 0]_x) on the left."""
    from scipy.linalg import expm
    rng = np.random.default_rng(5 + reject)
    p = orc.params(1, 1, 0, 0, r=3, T=1, k=1e-4, reject=reject)
    for _ in range(10):
        pts, Rtrue = random_points(rng, 49, outliers=4)
        R0 = rot(rng.normal(size=3), 0.2) @ Rtrue
        st0 = dict(tz=0.001, A=1.0, B=-0.5, C=2.0)
        out = orc.irls_step(pts, p, R0, st0["tz"], st0["A"], st0["B"], st0["C"])
        assert out["status"] == orc.OK
        eps, J = zip(*[orc.residual(R0, st0["tz"], st0["A"], st0["B"], st0["C"], q) for q in pts])
        eps, J = np.array(eps), np.array(J)
        mse = np.mean(eps ** 2)
        w = np.array([orc.weight(p, e, mse) for e in eps])
        assert np.array_equal(w, out["w"])
        sw = np.sqrt(w)
        b = np.linalg.lstsq(sw[:, None] * J, sw * eps, rcond=None)[0]
        assert np.allclose(out["b"], b, rtol=1e-8, atol=1e-12)
        assert out["tz"] == pytest.approx(st0["tz"] - b[2], abs=1e-12)
        assert out["A"] == pytest.approx(st0["A"] - b[3], rel=1e-9)
        assert out["B"] == pytest.approx(st0["B"] - b[4], rel=1e-9)
        assert out["C"] == pytest.approx(st0["C"] - b[5], rel=1e-9)
        assert np.allclose(out["R"], expm(skew([-b[0], -b[1], 0])) @ R0, atol=1e-12)


def test_irls_singular_system(orc):
    """All window points on one line: the curvature columns are dependent."""
    p = orc.params(1, 1, 0, 0, r=3, T=1)
    pts = np.c_[np.linspace(-0.02, 0.02, 20), np.zeros(20), np.zeros(20)]
    out = orc.irls_step(pts, p, np.eye(3), 0.0, 0.0, 0.0, 0.0)
    assert out["status"] == orc.SINGULAR


def test_irls_reaches_cauchy_minimum(orc):
    """Iterating Eq. iter_reweighted_update with Eq. weighting_function is IRLS
    for the Cauchy loss: after many iterations the state is a stationary point
    of sum_i k/2 ln(1 + eps_i^2/k), and an independent derivative-free
    minimiser (Nelder-Mead on an explicitly written residual) started from
    several points reaches the same parameters."""
    from scipy.optimize import minimize
    from scipy.linalg import expm
    rng = np.random.default_rng(11)
    k = 1e-4
    p = orc.params(1, 1, 0, 0, r=2, T=1, k=k)
    pts, Rtrue = random_points(rng, 25, noise=0.001, outliers=3)
    R0 = rot(rng.normal(size=3), 0.05) @ Rtrue
    R, tz, A, B, C = R0.copy(), 0.0, 0.0, 0.0, 0.0
    for _ in range(60):
        out = orc.irls_step(pts, p, R, tz, A, B, C)
        R, tz, A, B, C = out["R"], out["tz"], out["A"], out["B"], out["C"]
    assert np.abs(out["b"]).max() < 1e-10

    def cost(x):  # x = (theta_x, theta_y, tz, A, B, C) relative to R0
        Rx = expm(skew([x[0], x[1], 0])) @ R0
        loc = pts @ Rx.T
        e = x[3] / 2 * loc[:, 0] ** 2 + x[4] * loc[:, 0] * loc[:, 1] + x[5] / 2 * loc[:, 1] ** 2 - loc[:, 2] - x[2]
        return np.sum(k / 2 * np.log1p(e * e / k))

    # Composed x-y rotations carry some spin about the local z axis, which
    # the quadric absorbs (spinning the frame rotates [[A, B], [B, C]]), so
    # compare what is invariant: the cost, tz, the normal and k1, k2.
    k1o, k2o = orc.principal(A, B, C)
    for s in range(4):
        x0 = np.r_[0.0, 0.0, 0.0, A, B, C] * (s > 0) + rng.normal(size=6) * np.r_[0.02, 0.02, 1e-4, 1, 1, 1] * s
        r = minimize(cost, x0, method="Nelder-Mead",
                     options=dict(xatol=1e-11, fatol=1e-18, maxiter=60000, maxfev=60000))
        x = r.x
        assert r.fun == pytest.approx(np.sum(k / 2 * np.log1p(
            np.array([orc.residual(R, tz, A, B, C, q)[0] for q in pts]) ** 2 / k)), rel=1e-7)
        Rx = expm(skew([x[0], x[1], 0])) @ R0
        ev = np.linalg.eigvalsh([[x[3], x[4]], [x[4], x[5]]])
        assert ev[1] == pytest.approx(k1o, abs=1e-3 * (1 + abs(k1o)))
        assert ev[0] == pytest.approx(k2o, abs=1e-3 * (1 + abs(k1o)))
        assert np.allclose(Rx[2], R[2], atol=1e-5)
        assert x[2] == pytest.approx(tz, abs=1e-7)


# ---------------------------------------------------------------- step 8

def test_principal_vs_eigvalsh(orc):
    """Sec. 3.1.2: k1, k2 are the eigenvalues of the symmetric matrix
    [[A, B], [B, C]] of Eq. curv_tensor, largest first."""
    rng = np.random.default_rng(6)
    cases = [(10, 0, 10), (1, 2, 3), (0, 0, 0), (-5, 0, 5), (1e-8, 1e-8, 1e-8)]
    cases += [tuple(rng.normal(size=3) * 30) for _ in range(50)]
    for A, B, C in cases:
        k1, k2 = orc.principal(A, B, C)
        ev = np.linalg.eigvalsh(np.array([[A, B], [B, C]]))
        assert k1 == pytest.approx(ev[1], abs=1e-12 * (1 + abs(ev).max()))
        assert k2 == pytest.approx(ev[0], abs=1e-12 * (1 + abs(ev).max()))
        assert k1 >= k2


# ---------------------------------------------------------------- window

@pytest.mark.parametrize("r,stride", [(1, 1), (2, 1), (3, 1), (3, 2), (4, 3)])
def test_window_bruteforce(orc, r, stride):
    """Sec. 3.2: the fitted patch is the (2r+1)^2 square around the pixel (on
    a stride), clipped to the image, without pixels that have no range."""
    rng = np.random.default_rng(r * 10 + stride)
    H, W = 4, 5
    d = 1.0 + rng.random((H, W))
    d[rng.random((H, W)) < 0.3] = 0.0
    d[0, 0] = np.nan
    p = orc.params(1, 1, 0, 0, r=r, T=1, stride=stride)
    for v0, u0 in itertools.product(range(H), range(W)):
        got = {tuple(x) for x in orc.window(d, p, u0, v0)}
        want = set()
        for v in range(H):
            for u in range(W):
                du, dv = u - u0, v - v0
                if abs(du) <= r and abs(dv) <= r and du % stride == 0 and dv % stride == 0 \
                        and np.isfinite(d[v, u]) and d[v, u] > 0:
                    want.add((u, v))
        assert got == want


# ---------------------------------------------------------------- whole method

def test_plane_any_pose_has_zero_curvature(orc):
    """A plane has k1 = k2 = 0 and its own normal everywhere the window is
    fully on it (noise-free double-precision ranges)."""
    cam = synth.Camera(36, 44, 50.0, 50.0, 21.5, 17.5)
    for n in [(0, 0, 1), (0.4, -0.3, 1), (-0.8, 0.5, 1)]:
        nn = np.asarray(n, float) / np.linalg.norm(n)
        depth = plane_depth(cam, nn, 1.7)
        p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=4, T=3)
        f = orc.curvature_image(depth, p)
        assert (f.status == orc.OK).all()
        assert np.abs(f.k1).max() < 1e-8 and np.abs(f.k2).max() < 1e-8
        assert np.allclose(f.normal, nn, atol=1e-10)


def paraboloid_depth(cam, z0, a, c):
    """z = z0 + a X^2 + c Y^2 along each pixel ray, cancellation-free root"""
    rays = cam.rays()
    q = a * rays[..., 0] ** 2 + c * rays[..., 1] ** 2
    return 2 * z0 / (1 + np.sqrt(1 - 4 * q * z0))


@pytest.mark.parametrize("a,c", [(3.0, -5.0), (2.0, 2.0), (10.0, 0.0), (-4.0, -1.0)])
def test_paraboloid_apex(orc, a, c):
    """A paraboloid z = z0 + a X^2 + c Y^2 seen along its axis has curvatures
    (2a, 2c) at the apex (Eq. parabolic: A = d2z/dx2).  The symmetric window
    gives the exact normal, the data fit the model exactly, so one step lands
    on the answer and further steps stay there."""
    cam = synth.Camera(31, 31, 300.0, 300.0, 15.0, 15.0)
    depth = paraboloid_depth(cam, 1.2, a, c)
    for T in (1, 4):
        p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=7, T=T)
        res = orc.fit_pixel(depth, p, 15, 15)
        assert res.status == orc.OK
        k1, k2 = max(2 * a, 2 * c), min(2 * a, 2 * c)
        assert res.k1 == pytest.approx(k1, abs=1e-8)
        assert res.k2 == pytest.approx(k2, abs=1e-8)
        assert np.allclose(list(res.normal), [0, 0, 1], atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_rotated_paraboloid(orc, seed):
    """Curvature is invariant to a rigid motion of the surface: a paraboloid
    turned by up to 45 deg about its apex (which sits on a pixel ray) gives
    (2a, 2c) and the turned axis as the refined normal.  The initial normal is
    now only approximate, so this exercises the rotation part of the fit."""
    rng = np.random.default_rng(seed)
    cam = synth.Camera(41, 41, 400.0, 400.0, 20.0, 20.0)
    a, c = rng.uniform(1, 12), rng.uniform(-12, 12)
    Rs = synth._rand_rotation(rng, np.deg2rad(45))
    apex = 1.1 * np.array([(23 - cam.cx) / cam.fx, (18 - cam.cy) / cam.fy, 1.0])
    sad = synth.Saddle(apex, Rs, a, -c, 0.06)
    t, _, _, _ = sad.hit(cam.rays())
    depth = np.where(np.isfinite(t), t, 0.0)
    assert depth[18, 23] == pytest.approx(1.1, rel=1e-14)
    assert (depth[18 - 6:18 + 7, 23 - 6:23 + 7] > 0).all()
    p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=6, T=6)
    res = orc.fit_pixel(depth, p, 23, 18)
    assert res.status == orc.OK
    assert res.k1 == pytest.approx(max(2 * a, 2 * c), abs=1e-7)
    assert res.k2 == pytest.approx(min(2 * a, 2 * c), abs=1e-7)
    assert np.allclose(list(res.normal), Rs[:, 2], atol=1e-9)
    assert not np.allclose(list(res.n0), Rs[:, 2], atol=1e-6)


def sphere_apex_k(orc, rho, f, r=3, T=4):
    cam = synth.Camera(2 * r + 9, 2 * r + 9, f, f, r + 4.0, r + 4.0)
    t, _, _, _ = synth.Sphere(np.array([0.0, 0.0, 0.6 + rho]), rho).hit(cam.rays())
    depth = np.where(np.isfinite(t), t, 0.0)
    p = orc.params(cam.fx, cam.fy, cam.cx, cam.cy, r=r, T=T)
    res = orc.fit_pixel(depth, p, r + 4, r + 4)
    assert res.status == orc.OK
    return res.k1, res.k2


def test_sphere_bias_is_second_order(orc):
    """A sphere of radius rho has k1 = k2 = 1/rho.  Fitting a quadric over a
    window of half-width s leaves a bias of order (s/rho)^2 from the quartic
    term of the sphere; halving s (doubling f) divides it by about 4."""
    rho = 0.1
    errs = []
    for f in (400.0, 800.0, 1600.0):
        k1, k2 = sphere_apex_k(orc, rho, f)
        assert k1 == pytest.approx(k2, abs=1e-9)
        errs.append(abs(k1 - 1 / rho))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4
    assert errs[-1] < 2e-3 * (1 / rho)


def test_cylinder_apex(orc):
    """A cylinder of radius rho has principal curvatures (1/rho, 0)."""
    rho = 0.09
    for f, tol in ((800.0, 2e-3), (1600.0, 5e-4)):
        cam = synth.Camera(17, 17, f, f, 8.0, 8.0)
        cyl = synth.Cylinder(np.array([0.0, 0.0, 0.7 + rho]), np.array([0.0, 1.0, 0.0]), rho, 1.0)
        t, _, _, _ = cyl.hit(cam.rays())
        depth = np.where(np.isfinite(t), t, 0.0)
        p = orc.params(f, f, 8.0, 8.0, r=3, T=4)
        res = orc.fit_pixel(depth, p, 8, 8)
        assert res.status == orc.OK
        assert res.k1 == pytest.approx(1 / rho, rel=tol)
        assert abs(res.k2) < 1e-9


def test_invalid_pixels(orc):
    """Pixels without range, or without enough valid neighbours, are reported
    as invalid with NaN outputs."""
    p = orc.params(50.0, 50.0, 8.0, 8.0, r=3, T=2)
    f = orc.curvature_image(np.zeros((16, 16), np.float32), p)
    assert (f.status == orc.INVALID_CENTRE).all() and np.isnan(f.k1).all()
    d = np.zeros((16, 16))
    d[7:9, 7:9] = 1.0     # four points: a normal exists, but < 6 window points
    res = orc.fit_pixel(d, p, 7, 7)
    assert res.status == orc.FEW_POINTS and np.isnan(res.k1)


def test_float32_input_is_widened_exactly(orc):
    s = synth.sphere_scene(0)
    p = orc.params(*s.intrinsics, r=3, T=3)
    a = orc.curvature_image(s.depth, p, nthreads=2)
    b = orc.curvature_image(s.depth.astype(np.float64), p, nthreads=1)
    assert np.array_equal(a.k1, b.k1, equal_nan=True)
    assert np.array_equal(a.normal, b.normal, equal_nan=True)
    uv = np.array([[5, 5], [32, 24], [63, 47]])
    c = orc.curvature_pixels(s.depth, p, uv)
    assert np.array_equal(c.k1, a.k1[uv[:, 1], uv[:, 0]], equal_nan=True)
