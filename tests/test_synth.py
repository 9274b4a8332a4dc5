"""The input generator: seeded, shaped like the workloads, ground truth sane."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def test_seeded_and_shaped():
    a, b = synth.kinect_scene(3, H=120, W=160), synth.kinect_scene(3, H=120, W=160)
    assert np.array_equal(a.depth, b.depth)
    assert a.depth.dtype == np.float32 and a.depth.shape == (120, 160)
    c = synth.kinect_scene(4, H=120, W=160)
    assert not np.array_equal(a.depth, c.depth)
    assert a.cam.fx == pytest.approx(525 * 160 / 640)


def test_kinect_scene_statistics():
    s = synth.kinect_scene(0)
    z = s.depth
    frac0 = (z == 0).mean()
    assert 0.02 <= frac0 < 0.04          # 2 % blobs (+ a few misses)
    assert 0.3 < z[z > 0].min() and z.max() < 4.5
    assert len(s.prims) >= 12


def test_sphere_scene_ground_truth():
    s = synth.sphere_scene(0)
    assert s.depth.shape == (48, 64)
    assert s.gt_k1[24, 32] == pytest.approx(10.0) and s.gt_k2[24, 32] == pytest.approx(10.0)
    assert s.clean[24, 32] == pytest.approx(0.7)
    assert s.clean[0, 0] == pytest.approx(1.5)
    assert abs(float(s.depth[0, 0]) - 1.5) < 0.006    # 1 mm noise


def test_torus_hits_lie_on_the_surface_with_analytic_curvature():
    cam = synth.Camera(60, 80, 100.0, 100.0, 39.5, 29.5)
    tor = synth.Torus(np.array([0.0, 0.0, 0.8]), np.array([0.0, -0.6, -0.8]), 0.10, 0.03)
    z, k1, k2, n = tor.hit(cam.rays())
    ok = np.isfinite(z)
    assert ok.sum() > 100
    P = cam.rays() * np.where(ok, z, 0.0)[..., None]
    q = P - tor.c
    s = q @ tor.e
    dr = np.linalg.norm(q - s[..., None] * tor.e, axis=-1)
    assert np.abs(np.sqrt((dr - tor.R) ** 2 + s ** 2) - tor.rho)[ok].max() < 1e-12
    # tube curvature 1/rho everywhere; ring curvature between the inner and outer equators
    assert np.allclose(np.maximum(k1, k2)[ok], 1 / 0.03)
    assert k2[ok].min() >= -1 / 0.07 - 1e-9 and k2[ok].max() <= 1 / 0.13 + 1e-9
    assert np.allclose(np.linalg.norm(n[ok], axis=-1), 1.0)
