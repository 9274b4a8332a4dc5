"""The CUDA path against closed forms on the paper's synthetic objects
(Sec. 4.1, Table 1): a sphere of radius 0.10 m has k1 = k2 = 1/rho and a
cylinder of radius 0.09 m has (1/rho, 0).  A quadric fitted over a window of
half-width s on the surface keeps a bias of order (s/rho)^2 from the
surface's quartic terms (the oracle's own pin shows the second order on the
CPU), so each pixel whose whole window lies on the object and faces the camera
(n_z >= 0.7) must be within 0.5 (s/rho)^2 / rho of the closed form, with s
the window's half-diagonal on the surface, sqrt(2) r Z / (f n_z); and the
median error must grow by about (7/3)^2 from a 7 x 7 to a 15 x 15 window.
The same pixels also meet the parity rule against the oracle, and a noisy
torus (Table 1's third object) is one more parity case."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

PIVOT_TOL = 1e-5
F = 525.0


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1707_00385_gb300 import build
    build.build()
    import paper_1707_00385_gb300 as pc
    pc.load()
    return pc


def run_gpu(pc, scene, r, T=5):
    import torch
    c = pc.Curvature(*scene.intrinsics, window_radius=r, iterations=T)
    k1, k2, n = c(torch.from_numpy(np.ascontiguousarray(scene.depth, dtype=np.float32)).cuda())
    torch.cuda.synchronize()
    out = k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()
    c.close()
    return out


def interior(mask, r):
    """pixels whose whole (2r+1)^2 window lies inside mask"""
    m = mask.astype(np.int64)
    c = np.pad(m, ((1, 0), (1, 0))).cumsum(0).cumsum(1)
    H, W = m.shape
    y0, y1 = np.clip(np.arange(H) - r, 0, H), np.clip(np.arange(H) + r + 1, 0, H)
    x0, x1 = np.clip(np.arange(W) - r, 0, W), np.clip(np.arange(W) + r + 1, 0, W)
    return mask & ((c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0]) == (2 * r + 1) ** 2)


def object_crop(obj, rows=None, noise=None, seed=1):
    """The object in front of a wall at 1.5 m, 640 x 480 Kinect-like camera,
    cropped to the object's pixels plus a margin (rows limits the crop)."""
    cam = synth.kinect_camera(480, 640)
    wall = synth.Plane(np.array([0.0, 0.0, 1.0]), 1.5)
    sc = synth.render(cam, [obj, wall], noise=noise, rng=np.random.default_rng(seed))
    ys, xs = np.nonzero(sc.label == 0)
    y0, y1 = max(ys.min() - 8, 0), min(ys.max() + 9, 480)
    if rows is not None:
        y0, y1 = rows
    x0, x1 = max(xs.min() - 8, 0), min(xs.max() + 9, 640)
    c = synth.crop(sc, y0, x0, y1 - y0, x1 - x0)
    return c, sc.gt_normal[y0:y1, x0:x1]


SPHERE = synth.Sphere(np.array([0.0, 0.0, 0.8]), 0.10)
CYLINDER = synth.Cylinder(np.array([0.0, 0.0, 0.8]), np.array([0.0, 1.0, 0.0]), 0.09, 0.4)


@pytest.mark.parametrize("name,obj,rho,expect,rows", [
    ("sphere", SPHERE, 0.10, (10.0, 10.0), None),
    ("cylinder", CYLINDER, 0.09, (1 / 0.09, 0.0), (160, 320)),
])
def test_closed_form_within_second_order_bias(gpu, orc, name, obj, rho, expect, rows):
    from oracle import parity
    sc, gn = object_crop(obj, rows)
    med = {}
    for r in (3, 7):
        k1, k2, n = run_gpu(gpu, sc, r)
        nz = np.abs(gn[..., 2])
        m = interior(sc.label == 0, r) & np.isfinite(k1) & (nz >= 0.7)
        assert m.sum() > 2000
        s = np.sqrt(2.0) * r * sc.depth[m] / F / nz[m]
        bound = 0.5 * (s / rho) ** 2 / rho
        e1, e2 = np.abs(k1[m] - expect[0]), np.abs(k2[m] - expect[1])
        print(name, r, "max err / bound", float((e1 / bound).max()), float((e2 / bound).max()))
        assert np.all(e1 <= bound) and np.all(e2 <= bound)
        med[r] = float(np.median(e1))
        # the same pixels against the oracle: noise-free, so the iterations
        # settle; on the 7 x 7 cylinder window the probe's coordinate noise
        # still moves a tenth of the answers by over a quarter of the
        # tolerance (GB300: 0.894 gated, every pixel within 0.01 of it)
        uv = np.stack(np.nonzero(m)[::-1], 1).astype(np.int32)
        p = orc.params(*sc.intrinsics, r=r, T=5, pivot_tol=PIVOT_TOL)
        ref = parity.reference(sc.depth, p, uv=uv)
        rep = parity.compare(k1[m], k2[m], n[m], ref, pivot_tol=PIVOT_TOL)
        print(rep.summary())
        assert rep.ok() and rep.n_well_posed >= 0.87 * rep.n_valid_oracle, rep.summary()
        assert rep.frac_within_tol_all >= 0.99, rep.summary()
    ratio = med[7] / med[3]
    print(name, "median error r=3", med[3], "r=7", med[7], "ratio", ratio)
    assert 3.5 < ratio < 7.0        # (7/3)^2 = 5.4: second order in the window size


def test_torus_scene_parity(gpu, orc):
    """The 10 cm / 3 cm torus of Table 1 with Kinect-like noise, window radius
    7, 5 iterations, against the oracle (every pixel of the crop)."""
    from oracle import parity
    torus = synth.Torus(np.array([0.0, 0.0, 0.8]), np.array([0.0, -0.6, -0.8]), 0.10, 0.03)
    sc, _ = object_crop(torus, noise=synth.kinect_noise)
    k1, k2, n = run_gpu(gpu, sc, 7)
    p = orc.params(*sc.intrinsics, r=7, T=5, pivot_tol=PIVOT_TOL)
    rep = parity.compare(k1, k2, n, parity.reference(sc.depth, p), pivot_tol=PIVOT_TOL)
    print(rep.summary())
    case = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    print("PARITY_ROW " + json.dumps({"case": case, **rep.row()}))
    assert rep.ok(), rep.summary()
    assert rep.n_well_posed >= 0.56 * rep.n_valid_oracle, rep.summary()     # GB300: 0.585
    assert rep.frac_within_tol_all >= 0.77, rep.summary()                    # GB300: 0.789
    # at least as many as the oracle with single-precision sums (GB300: 0.780)
    assert rep.frac_within_tol_all >= rep.frac_within_tol_f32_sums - 0.005, rep.summary()
    assert rep.max_normal_angle_well_posed < 1e-4, rep.summary()


@pytest.mark.parametrize("r", [3, 7])
def test_tilted_plane_has_zero_curvature(gpu, orc, r):
    """The degenerate case of the shape operator: a noise-free tilted plane
    (no curvature, so both eigenvalues 0 and T2 = hypot(0, 0)).  The only
    error is the rounding of the stored ranges (about 1e-7 m), far below
    0.05 m^-1 of curvature and 3e-5 rad of normal over the window; the oracle
    agrees under the parity rule."""
    from oracle import parity
    n_true = np.array([0.3, -0.2, 1.0])
    n_true /= np.linalg.norm(n_true)
    cam = synth.kinect_camera(480, 640)
    sc = synth.crop(synth.render(cam, [synth.Plane(n_true, 1.2)]), 200, 270, 70, 100)
    k1, k2, n = run_gpu(gpu, sc, r)
    m = interior(sc.label == 0, r)
    assert m.sum() > 3000 and np.isfinite(k1[m]).all() and np.isfinite(k2[m]).all()
    print("plane r", r, "max |k|", float(np.abs(k1[m]).max()), float(np.abs(k2[m]).max()))
    assert np.abs(k1[m]).max() < 0.05 and np.abs(k2[m]).max() < 0.05
    # angle by atan2(|n x t|, |n . t|): arccos of a dot product of single-precision
    # unit vectors is only good to about sqrt(2e-7) = 4.5e-4 rad near zero
    nm = n[m].astype(np.float64)
    ang = np.arctan2(np.linalg.norm(np.cross(nm, n_true), axis=1), np.abs(nm @ n_true))
    print("plane r", r, "max normal angle", float(ang.max()))
    assert ang.max() < 3e-5, float(ang.max())      # range rounding 1e-7 m over a window of 7 mm: 1e-5 rad
    p = orc.params(*sc.intrinsics, r=r, T=5, pivot_tol=PIVOT_TOL)
    rep = parity.compare(k1, k2, n, parity.reference(sc.depth, p), pivot_tol=PIVOT_TOL)
    print(rep.summary())
    assert rep.ok(), rep.summary()
