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
