"""Pins of the oracle's organised outputs (point cloud and initial-normal
field, Sec. 3 and Sec. 3.2.1): they must equal the per-pixel oracle functions
that the other pins fix, and reproduce closed forms."""
import numpy as np

import synth


def test_backproject_image_is_the_pinhole_inverse(orc):
    rng = np.random.default_rng(3)
    H, W = 13, 17
    z = rng.uniform(0.5, 3.0, (H, W)).astype(np.float32)
    z[2, 3] = 0.0
    z[5, 7] = np.nan
    z[8, 1] = -1.0
    z[9, 9] = np.inf
    p = orc.params(400.0, 410.0, 8.2, 6.1, r=3, T=0)
    xyz = orc.backproject_image(z, p)
    bad = ~(np.isfinite(z) & (z > 0))
    assert np.isnan(xyz[bad]).all() and np.isfinite(xyz[~bad]).all()
    v, u = np.nonzero(~bad)
    zz = z[v, u].astype(np.float64)
    # projecting back gives the pixel centres, and the third coordinate is the range
    assert np.allclose(400.0 * xyz[v, u, 0] / zz + 8.2, u, atol=1e-12)
    assert np.allclose(410.0 * xyz[v, u, 1] / zz + 6.1, v, atol=1e-12)
    assert np.array_equal(xyz[v, u, 2], zz)
    for (uu, vv) in [(0, 0), (16, 12), (4, 7)]:
        assert np.array_equal(xyz[vv, uu], orc.backproject(p, uu, vv, float(z[vv, uu])))


def test_initial_normal_image_matches_the_per_pixel_oracle(orc):
    s = synth.crop(synth.kinect_scene(5, invalid_frac=0.05), 100, 150, 24, 30)
    p = orc.params(*s.intrinsics, r=3, T=0)
    n, st = orc.initial_normal_image(s.depth, p)
    d = s.depth.astype(np.float64)
    for v in range(s.depth.shape[0]):
        for u in range(s.depth.shape[1]):
            if not (s.depth[v, u] > 0):
                assert st[v, u] == orc.INVALID_CENTRE and np.isnan(n[v, u]).all()
                continue
            s2, n2 = orc.initial_normal(d, p, u, v)
            assert st[v, u] == s2
            if s2 == orc.OK:
                assert np.array_equal(n[v, u], n2)
            else:
                assert np.isnan(n[v, u]).all()


def test_initial_normal_image_of_a_plane_is_exact(orc):
    cam = synth.kinect_camera(40, 48)
    nrm = np.array([0.3, -0.2, 1.0])
    nrm /= np.linalg.norm(nrm)
    sc = synth.render(cam, [synth.Plane(nrm, 1.2)], noise=None)
    p = orc.params(*sc.intrinsics, r=3, T=0)
    n, st = orc.initial_normal_image(sc.depth.astype(np.float32), p)
    ok = st == orc.OK
    assert ok.sum() == sc.depth.size
    # the rendered ranges are rounded to float32: the fitted plane is exact to that rounding
    expect = nrm   # n_z > 0: (-a, -b, 1) of z = a x + b y + c
    ang = np.degrees(np.arccos(np.clip(n[ok] @ expect, -1, 1)))
    assert ang.max() < 1e-3


def test_sensitivity_of_the_normal_field_flags_near_singular_patches(orc):
    from oracle import parity
    s = synth.crop(synth.kinect_scene(6), 200, 300, 24, 32)
    p = orc.params(*s.intrinsics, r=3, T=0)
    ref = parity.normal_reference(s.depth, p)
    ok = ref.status == orc.OK
    assert np.isfinite(ref.sens[ok]).mean() > 0.99
    # the perturbations are tiny: most normals move by far less than the tolerance
    assert np.median(ref.sens[ok]) < 1e-6
    # a planted rotation of the oracle's own field is caught by the comparison
    bad = ref.normal.copy()
    bad[ok] = bad[ok] @ np.array([[1, 0, 0], [0, np.cos(1e-3), -np.sin(1e-3)], [0, np.sin(1e-3), np.cos(1e-3)]]).T
    rep = parity.compare_normals(bad, ref)
    assert not rep.ok() and rep.n_well_posed_bad > 0
    assert parity.compare_normals(ref.normal, ref).ok()
