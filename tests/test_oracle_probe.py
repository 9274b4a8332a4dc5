"""The oracle's sensitivity probe, on which the parity rule decides which
pixels are determined at single precision: off, it changes nothing; on, it is
reproducible from its seed, moves each entry of the normal equations by at
most a times the bound of its sum of term magnitudes (keeping them
symmetric), its amplitude has the size of the error that single-precision
sums actually make (measured with the oracle's f32_sums mode), and it flags
the pixels whose answer is not fixed at single precision -- none where the
iteration has settled on a noise-free sphere, some but not all of a noisy
Kinect-like crop."""
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
    """Entry (a, c) of the normal matrix moves by at most a sqrt(N_aa N_cc),
    entry a of the right-hand side by at most a sqrt(N_aa E), E = sum w eps^2
    (the Cauchy-Schwarz bounds of the sums of term magnitudes)."""
    rng = np.random.default_rng(5)
    pts = rng.normal(scale=0.02, size=(49, 3))
    pts[:, 2] = 3.0 * pts[:, 0] ** 2 - 2.0 * pts[:, 1] ** 2 + 1e-4 * rng.standard_normal(49)
    R = np.eye(3)
    state = (0.0, 1.0, 0.5, -2.0)
    p0 = orc.params(500.0, 500.0, 0.0, 0.0, r=3, T=1)
    ref = orc.irls_step(pts, p0, R, *state)
    eps = np.array([orc.residual(R, *state, q)[0] for q in pts])
    E = np.sum(ref["w"] * eps * eps)
    d = np.sqrt(np.diag(ref["N"]))
    a = 1e-3
    for seed in (1, 2, 3):
        q = orc.params(500.0, 500.0, 0.0, 0.0, r=3, T=1, perturb=a, perturb_seed=seed)
        got = orc.irls_step(pts, q, R, *state)
        x = (got["N"] - ref["N"]) / np.outer(d, d)
        assert np.all(np.abs(x) <= a * (1 + 1e-9)) and np.any(np.abs(x) > a / 100)
        # one noise value per unordered pair (a, c): the perturbed matrix stays symmetric
        assert np.allclose(got["N"], got["N"].T, rtol=0, atol=1e-14 * np.abs(ref["N"]).max())
        y = (got["rhs"] - ref["rhs"]) / (d * np.sqrt(E))
        assert np.all(np.abs(y) <= a * (1 + 1e-9)) and np.any(y != 0.0)


def _scaled_sum_errors(orc, depth, p, pixels):
    """Root mean square, in units of sqrt(N) u, of the error that sums in
    single precision make (the oracle's f32_sums mode against its double
    sums, at the same states along each pixel's own iteration), each entry
    scaled as the probe scales its noise: normal matrix, right-hand side."""
    q = copy.copy(p)
    q.f32_sums = 1
    d64 = depth.astype(np.float64)
    en, er = [], []
    for u, v in pixels:
        st, nrm = orc.initial_normal(d64, p, u, v)
        if st != orc.OK:
            continue
        uv = orc.window(d64, p, u, v)
        P0 = orc.backproject(p, u, v, d64[v, u])
        pts = np.array([orc.backproject(p, a, b, d64[b, a]) for a, b in uv]) - P0
        R, tz, A, B, C = orc.frame_from_normal(nrm), 0.0, 0.0, 0.0, 0.0
        for _ in range(p.T):
            s64 = orc.irls_step(pts, p, R, tz, A, B, C)
            s32 = orc.irls_step(pts, q, R, tz, A, B, C)
            eps = np.array([orc.residual(R, tz, A, B, C, x)[0] for x in pts])
            E = np.sum(s64["w"] * eps * eps)
            dg = np.sqrt(np.diag(s64["N"]))
            iu = np.triu_indices(6)
            en.append((np.abs(s32["N"] - s64["N"]) / np.outer(dg, dg))[iu])
            er.append(np.abs(s32["rhs"] - s64["rhs"]) / (dg * np.sqrt(E)))
            if s64["status"] != orc.OK:
                break
            R, tz, A, B, C = s64["R"], s64["tz"], s64["A"], s64["B"], s64["C"]
    unit = np.sqrt(parity.window_points(p)) * parity.U
    rms = lambda x: float(np.sqrt(np.mean(np.concatenate(x) ** 2))) / unit
    return rms(en), rms(er)


@pytest.mark.parametrize("r", [3, 7])
def test_probe_amplitude_is_calibrated_on_single_precision_sums(orc, r):
    """The probe's noise has the size of real single-precision summation error:
    its root mean square a / sqrt(3) covers the measured one (scaled units),
    without exceeding it by more than a factor 3."""
    sc = synth.kinect_scene(0)
    rng = np.random.default_rng(11)
    pix = [(int(rng.integers(r, 640 - r)), int(rng.integers(r, 480 - r))) for _ in range(80)]
    p = orc.params(*sc.intrinsics, r=r, T=5)
    rms_n, rms_r = _scaled_sum_errors(orc, sc.depth, p, pix)
    probe_rms = parity.PROBE_C / np.sqrt(3.0)
    assert rms_n <= probe_rms <= 3.0 * rms_n, (rms_n, probe_rms)
    assert rms_r <= probe_rms


def test_regression_probe_amplitude_is_calibrated_on_single_precision_sums(orc):
    """The same for the sums of the initial-normal regression (49 points)."""
    sc = synth.kinect_scene(3)
    p = orc.params(*sc.intrinsics, r=3, T=0)
    q = copy.copy(p)
    q.f32_sums = 1
    d64 = sc.depth.astype(np.float64)
    rng = np.random.default_rng(12)
    em, ev = [], []
    for _ in range(600):
        u, v = int(rng.integers(0, 640)), int(rng.integers(0, 480))
        c, s64 = orc.regression_sums(d64, p, u, v)
        _, s32 = orc.regression_sums(d64, q, u, v)
        if c < 3 or not d64[v, u] > 0:
            continue
        m00, m01, m11, v0, v1, szz = s64
        scale = np.array([m00, np.sqrt(m00 * m11), m11, np.sqrt(m00 * szz), np.sqrt(m11 * szz)])
        e = np.abs(s32[:5] - s64[:5]) / scale
        if np.all(np.isfinite(e)):
            em.append(e[:3])
            ev.append(e[3:])
    unit = 7.0 * parity.U
    rms_m = float(np.sqrt(np.mean(np.concatenate(em) ** 2))) / unit
    rms_v = float(np.sqrt(np.mean(np.concatenate(ev) ** 2))) / unit
    probe_rms = parity.PROBE_C / np.sqrt(3.0)
    assert rms_m <= probe_rms <= 3.0 * rms_m, (rms_m, probe_rms)
    assert rms_v <= probe_rms


def test_single_precision_sums_change_the_answer_only_by_rounding(orc, noisy):
    """The calibration mode is the method with its sums rounded: on a settled
    noise-free sphere it agrees with the double-precision oracle to a small
    fraction of the tolerance, and on a noisy crop it moves some pixels."""
    s = synth.sphere_scene(0)
    clean = np.where(np.isfinite(s.clean), s.clean, 0.0).astype(np.float32)
    p = orc.params(*s.intrinsics, r=3, T=8)
    f = orc.curvature_image(clean, p)
    q = copy.copy(p)
    q.f32_sums = 1
    g = orc.curvature_image(clean, q)
    settled = f.converged() & (s.label == 0) & (g.status == orc.OK)
    assert settled.sum() > 20
    assert np.max(np.abs(g.k1 - f.k1)[settled] / parity.tolerance(f.k1[settled])) < 0.05
    p = orc.params(*noisy.intrinsics, r=7, T=5)
    q = copy.copy(p)
    q.f32_sums = 1
    f, g = orc.curvature_image(noisy.depth, p), orc.curvature_image(noisy.depth, q)
    both = (f.status == orc.OK) & (g.status == orc.OK)
    assert np.any(g.k1[both] != f.k1[both])


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


def test_tensor_core_moments_need_the_split(orc, noisy):
    """The accuracy side of forming J^T W J on tensor cores (a design
    question, not the method): with one TF32 product per term far fewer
    pixels of a noisy crop stay within the parity tolerance of the FP64
    oracle than with single-precision sums, while the three-product split
    keeps them at the single-precision level."""
    p = orc.params(*noisy.intrinsics, r=7, T=5)
    f = orc.curvature_image(noisy.depth, p)
    within = {}
    for mode in (1, 2, 3):
        q = copy.copy(p)
        q.f32_sums = mode
        g = orc.curvature_image(noisy.depth, q)
        both = (f.status == orc.OK) & (g.status == orc.OK)
        rel = np.maximum(np.abs(g.k1 - f.k1) / parity.tolerance(f.k1), np.abs(g.k2 - f.k2) / parity.tolerance(f.k2))
        within[mode] = float(np.mean(rel[both] <= 1))
    assert within[2] < within[1] - 0.1, within
    assert abs(within[3] - within[1]) < 0.02, within


def test_reference_reports_the_single_precision_sums_floor(orc):
    """parity.reference keeps, beside the spread, how many pixels the oracle
    itself keeps within tolerance when its sums are formed in single precision
    (the yardstick a single-precision kernel is read against): the same
    fraction as a direct comparison of the two oracle runs."""
    from oracle import parity
    import synth
    s = synth.crop(synth.kinect_scene(0), 180, 250, 24, 40)
    p = orc.params(*s.intrinsics, r=5, T=5, pivot_tol=1e-5)
    ref = parity.reference(s.depth, p)
    f = orc.curvature_image(s.depth, p)
    q = orc.params(*s.intrinsics, r=5, T=5, pivot_tol=1e-5)
    q.f32_sums = 1
    g = orc.curvature_image(s.depth, q)
    both = (f.status == orc.OK) & (g.status == orc.OK)
    rel = np.maximum(np.abs(g.k1 - f.k1) / parity.tolerance(f.k1), np.abs(g.k2 - f.k2) / parity.tolerance(f.k2))
    assert both.sum() > 500
    assert ref.f32_within == float(np.mean(rel[both] <= 1))
    assert 0.5 < ref.f32_within < 1.0          # single-precision sums do move some answers
