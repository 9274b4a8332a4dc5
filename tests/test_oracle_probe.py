"""The oracle's sensitivity probe, on which the parity rule decides which
pixels are determined at single precision: off, it changes nothing; on, it is
reproducible from its seed, scales each entry of the normal equations by a
factor within 1 +- a (keeping them symmetric), and flags the pixels whose
answer is not fixed at single precision -- none where the iteration has
settled on a noise-free sphere, some but not all of a noisy Kinect-like crop."""
import copy

import numpy as np
import pytest

import synth
from oracle import parity

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def noisy():
    return synth.crop(synth.kinect_scene(3), 150, 250, 24, 40)


def run(orc, depth, p, **probe):
    q = copy.copy(p)
    for k, v in probe.items():
        setattr(q, k, v)
    return orc.curvature_image(depth, q, nthreads=1)


def same(a, b):
    return (np.array_equal(a.k1, b.k1, equal_nan=True) and np.array_equal(a.k2, b.k2, equal_nan=True)
            and np.array_equal(a.normal, b.normal, equal_nan=True) and np.array_equal(a.status, b.status))


def test_probe_off_changes_nothing(orc, noisy):
    p = orc.params(*noisy.intrinsics, r=5, T=5)
    base = run(orc, noisy.depth, p)
    assert same(base, run(orc, noisy.depth, p, perturb_seed=12345))
    assert same(base, run(orc, noisy.depth, p, perturb=0.0, perturb_points=0.0, perturb_seed=7))


def test_probe_is_reproducible_from_its_seed(orc, noisy):
    p = orc.params(*noisy.intrinsics, r=5, T=5)
    a = run(orc, noisy.depth, p, perturb=1e-6, perturb_points=1e-6, perturb_seed=3)
    b = run(orc, noisy.depth, p, perturb=1e-6, perturb_points=1e-6, perturb_seed=3)
    c = run(orc, noisy.depth, p, perturb=1e-6, perturb_points=1e-6, perturb_seed=4)
    assert same(a, b)
    ok = (a.status == 0) & (c.status == 0)
    assert np.any(a.k1[ok] != c.k1[ok])


def test_probe_scales_normal_equations_within_bounds(orc):
    rng = np.random.default_rng(5)
    pts = rng.normal(scale=0.02, size=(49, 3))
    pts[:, 2] = 3.0 * pts[:, 0] ** 2 - 2.0 * pts[:, 1] ** 2 + 1e-4 * rng.standard_normal(49)
    R = np.eye(3)
    p0 = orc.params(500.0, 500.0, 0.0, 0.0, r=3, T=1)
    ref = orc.irls_step(pts, p0, R, 0.0, 1.0, 0.5, -2.0)
    a = 1e-3
    for seed in (1, 2, 3):
        q = orc.params(500.0, 500.0, 0.0, 0.0, r=3, T=1, perturb=a, perturb_seed=seed)
        got = orc.irls_step(pts, q, R, 0.0, 1.0, 0.5, -2.0)
        assert np.all(ref["N"] != 0)
        f = got["N"] / ref["N"]
        assert np.all(np.abs(f - 1.0) <= a) and np.any(np.abs(f - 1.0) > a / 100)
        # one factor per unordered pair (a, c): the perturbed matrix stays symmetric
        assert np.allclose(f, f.T, rtol=0, atol=1e-14)
        fr = got["rhs"] / ref["rhs"]
        assert np.all(np.abs(fr - 1.0) <= a) and np.any(fr != 1.0)


def test_probe_leaves_settled_pixels_determined(orc):
    """Where the fixed-count iteration has settled (its last update is tiny)
    on a noise-free sphere, rounding-sized noise cannot move the answer by a
    quarter of the tolerance."""
    s = synth.sphere_scene(0)
    clean = np.where(np.isfinite(s.clean), s.clean, 0.0).astype(np.float32)
    p = orc.params(*s.intrinsics, r=3, T=8)
    ref = parity.reference(clean, p, nthreads=1)
    settled = ref.field.converged() & (s.label == 0)
    assert settled.sum() > 20
    assert ref.sens[settled].max() <= 0.25


def test_probe_flags_some_but_not_all_noisy_pixels(orc, noisy):
    p = orc.params(*noisy.intrinsics, r=7, T=5)
    ref = parity.reference(noisy.depth, p, nthreads=1)
    valid = ref.field.status == 0
    flagged = np.mean(ref.sens[valid] > 0.25)
    assert 0.0 < flagged < 0.8, flagged
