"""CUDA path (through the C ABI) against the FP64 oracle, element by element,
on seeded synthetic range images.

Rule (oracle/parity.py): |dk| <= 1e-4 + 1e-4 |k| for k1 and k2 on every
well-posed pixel (the oracle's own answer is fixed to a quarter of that
tolerance under single-precision-sized perturbation); validity agrees except
at the singularity threshold; NaN patterns of k1, k2 and the normal agree.
Each case also has a floor on the well-posed fraction and on the fraction of
all pixels within tolerance, each about two points under the value measured
on a GB300, so a regression cannot hide behind the rule."""
import json
import os

import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

PIVOT_TOL = 1e-5
# The oracle itself, with its sums formed in single precision (plain loop
# order, everything else FP64), keeps a fraction of the pixels within the
# tolerance; the CUDA path must keep at least as many, up to this slack (GB300:
# at or above it in every case but the 64-iteration one, 0.0012 below).
F32_SLACK = 0.005


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


def run_gpu(pc, depth, intr, r, T, **params):
    import torch
    c = pc.Curvature(*intr, window_radius=r, iterations=T, **params)
    d = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.float32)).cuda()
    k1, k2, n = c(d)
    torch.cuda.synchronize()
    out = k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()
    c.close()
    return out


def check(pc, orc, scene, r, T, min_well_posed, min_within, uv=None, **params):
    from oracle import parity
    k1, k2, n = run_gpu(pc, scene.depth, scene.intrinsics, r, T, **params)
    okw = {("rn" if k == "normal_radius" else k): v for k, v in params.items()}
    p = orc.params(*scene.intrinsics, r=r, T=T, pivot_tol=PIVOT_TOL, **okw)
    ref = parity.reference(scene.depth, p, nthreads=0, uv=uv)
    if uv is not None:
        k1, k2, n = k1[uv[:, 1], uv[:, 0]], k2[uv[:, 1], uv[:, 0]], n[uv[:, 1], uv[:, 0]]
    rep = parity.compare(k1, k2, n, ref, pivot_tol=PIVOT_TOL)
    print(rep.summary())
    case = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    print("PARITY_ROW " + json.dumps({"case": case, **rep.row()}))
    assert rep.nan_pattern_ok
    assert rep.n_validity_mismatch == 0, rep.summary()
    assert rep.n_well_posed_bad == 0, rep.summary()
    assert rep.n_well_posed >= min_well_posed * rep.n_valid_oracle, rep.summary()
    assert rep.frac_within_tol_all >= min_within, rep.summary()
    assert rep.frac_within_tol_all >= rep.frac_within_tol_f32_sums - F32_SLACK, rep.summary()
    assert rep.max_normal_angle_well_posed < 1e-4, rep.summary()
    return rep


@pytest.fixture(scope="module")
def kinect640():
    return synth.kinect_scene(0)


@pytest.fixture(scope="module")
def crop(kinect640):
    # 70 x 100: several 32 x 8 tiles and a ragged tail in both directions
    return synth.crop(kinect640, 180, 250, 70, 100)


def test_sphere_scene_64x48(gpu, orc):
    """64 x 48 sphere (r = 0.10 m at 0.80 m) in front of a plane, 1 mm noise,
    window radius 3, 3 iterations, whole image."""
    check(gpu, orc, synth.sphere_scene(0), 3, 3, min_well_posed=0.89, min_within=0.92)


@pytest.mark.parametrize("r,floor,within", [(3, 0.81, 0.955), (6, 0.74, 0.93), (7, 0.71, 0.91), (11, 0.61, 0.875),
                                             (12, 0.60, 0.87)])
def test_kinect_crop_radii(gpu, orc, crop, r, floor, within):
    # larger windows mix more surfaces and settle more slowly: fewer pixels
    # have an answer fixed at single precision after 5 iterations
    check(gpu, orc, crop, r, 5, min_well_posed=floor, min_within=within)


def test_kinect_crop_sparse_window(gpu, orc, crop):
    """Strided window (run-time radius path): 15 x 15 sampled every 2 pixels."""
    check(gpu, orc, crop, 7, 5, min_well_posed=0.83, min_within=0.925, stride=2)


def test_kinect_crop_runtime_radius(gpu, orc, crop):
    """Radius 15, beyond the unrolled instantiations, 3 iterations."""
    check(gpu, orc, crop, 15, 3, min_well_posed=0.52, min_within=0.845)


def test_kinect_crop_rejection(gpu, orc, crop):
    """The rejection filter of the weighting function (weight 0 above 2 MSE)."""
    check(gpu, orc, crop, 7, 5, min_well_posed=0.80, min_within=0.94, reject=1)


def test_kinect_crop_other_k_and_normal_radius(gpu, orc, crop):
    check(gpu, orc, crop, 5, 4, min_well_posed=0.75, min_within=0.94, k=4e-4, normal_radius=2)


def test_kinect_crop_largest_normal_radius(gpu, orc, crop):
    """PC_MAX_NORMAL_RADIUS (17 x 17 initial-normal patch) around a 7 x 7
    window: the staged halo is set by the normal patch, not the window."""
    check(gpu, orc, crop, 3, 5, min_well_posed=0.80, min_within=0.94,     # GB300: 0.823, 0.964
          normal_radius=gpu.pcurv.PC_MAX_NORMAL_RADIUS)


def test_full_frame_sampled(gpu, orc, kinect640):
    """640 x 480, radius 7, 5 iterations (the benchmark's launch): 2500 random
    pixels plus two whole 32 x 8 tiles (a corner and an interior one)."""
    rng = np.random.default_rng(7)
    uv = np.stack([rng.integers(0, 640, 2500), rng.integers(0, 480, 2500)], 1)
    tiles = [np.stack(np.meshgrid(np.arange(u0, u0 + 32), np.arange(v0, v0 + 8)), -1).reshape(-1, 2)
             for u0, v0 in ((0, 0), (320, 240))]
    uv = np.concatenate([uv] + tiles).astype(np.int32)
    check(gpu, orc, kinect640, 7, 5, min_well_posed=0.74, min_within=0.935, uv=uv)


def test_full_frame_every_pixel_batched(gpu, orc, kinect640):
    """Every pixel of one 640 x 480 frame, r = 7, T = 5, computed by the
    persistent batch kernel the benchmark times (pc_compute_batch)."""
    import torch
    c = gpu.Curvature(*kinect640.intrinsics, window_radius=7, iterations=5)
    d = torch.from_numpy(kinect640.depth).cuda()
    out = (torch.empty_like(d), torch.empty_like(d), torch.empty(d.shape + (3,), device="cuda"))
    c.batch([(d, kinect640.intrinsics) + out])
    torch.cuda.synchronize()
    c.close()
    from oracle import parity
    k1, k2, n = (t.cpu().numpy() for t in out)
    p = orc.params(*kinect640.intrinsics, r=7, T=5, pivot_tol=PIVOT_TOL)
    rep = parity.compare(k1, k2, n, parity.reference(kinect640.depth, p), pivot_tol=PIVOT_TOL)
    print(rep.summary())
    case = os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0]
    print("PARITY_ROW " + json.dumps({"case": case, **rep.row()}))
    assert rep.ok(), rep.summary()
    assert rep.n_well_posed >= 0.72 * rep.n_valid_oracle, rep.summary()     # 0.745 of the oracle's pixels
    assert rep.frac_within_tol_all >= 0.93, rep.summary()                    # GB300: 0.940
    assert rep.frac_within_tol_all >= rep.frac_within_tol_f32_sums - F32_SLACK, rep.summary()   # 0.931
    assert rep.max_normal_angle_well_posed < 1e-4, rep.summary()


def test_tof_scene_512x424(gpu, orc):
    """Time-of-flight noise model at 512 x 424 (sampled pixels)."""
    s = synth.kinect_scene(3, H=424, W=512, noise="tof")
    rng = np.random.default_rng(3)
    uv = np.stack([rng.integers(0, 512, 1500), rng.integers(0, 424, 1500)], 1).astype(np.int32)
    check(gpu, orc, s, 7, 5, min_well_posed=0.85, min_within=0.93, uv=uv)


def test_noise_free_scene_all_pixels_close(gpu, orc):
    """Without noise almost every pixel converges and must match."""
    s = synth.crop(synth.kinect_scene(1, noise="none", invalid_frac=0.0), 200, 200, 48, 80)
    check(gpu, orc, s, 7, 5, min_well_posed=0.98, min_within=0.98)


def test_closed_form_paraboloid_on_gpu(gpu):
    """A paraboloid z = z0 + a X^2 + c Y^2 seen along its axis: (2a, 2c) at the
    apex (float32 ranges, so to a few 1e-4 relative)."""
    cam = synth.Camera(31, 31, 300.0, 300.0, 15.0, 15.0)
    rays = cam.rays()
    a, c, z0 = 3.0, -5.0, 1.2
    q = a * rays[..., 0] ** 2 + c * rays[..., 1] ** 2
    depth = (2 * z0 / (1 + np.sqrt(1 - 4 * q * z0))).astype(np.float32)
    k1, k2, n = run_gpu(gpu, depth, (300.0, 300.0, 15.0, 15.0), 7, 4)
    assert k1[15, 15] == pytest.approx(6.0, rel=2e-3)
    assert k2[15, 15] == pytest.approx(-10.0, rel=2e-3)
    assert np.allclose(n[15, 15], [0, 0, 1], atol=1e-5)


@pytest.fixture(scope="module")
def small_crop(kinect640):
    # 40 x 48: two tile rows with a ragged tail, small enough for the largest windows
    return synth.crop(kinect640, 200, 300, 40, 48)


def test_largest_window_radius(gpu, orc, small_crop):
    """PC_MAX_RADIUS = 24 (49 x 49 window), 2 iterations.  Parity is not
    claimed for this window on this crop: its windows span several surfaces
    and even 12 iterations leave most pixels unsettled, so under
    single-precision-sized noise the oracle's own answer moves for all but
    about 14 % of them.  The case still checks those pixels, validity and the
    NaN patterns, and floors the fraction of all pixels within tolerance."""
    import paper_1707_00385_gb300 as pc
    r = pc.pcurv.PC_MAX_RADIUS
    check(gpu, orc, small_crop, r, 2, min_well_posed=0.12, min_within=0.75)


def test_paper_sparse_37x37_window(gpu, orc, crop):
    """The paper's sparsely sampled 37 x 37 patch: radius 18 sampled every 3 pixels."""
    check(gpu, orc, crop, 18, 5, min_well_posed=0.74, min_within=0.88, stride=3)


def test_most_iterations(gpu, orc, small_crop):
    """PC_MAX_ITERATIONS = 64 at radius 3: the iterations settle, so most pixels are
    fixed at single precision again."""
    import paper_1707_00385_gb300 as pc
    check(gpu, orc, small_crop, 3, pc.pcurv.PC_MAX_ITERATIONS, min_well_posed=0.76, min_within=0.92)


def test_no_iterations(gpu, orc, crop):
    """T = 0: curvatures 0, normal = the initial normal, validity from the
    normal and the window count."""
    from oracle import parity
    k1, k2, n = run_gpu(gpu, crop.depth, crop.intrinsics, 7, 0)
    p = orc.params(*crop.intrinsics, r=7, T=0, pivot_tol=PIVOT_TOL)
    f = orc.curvature_image(crop.depth, p)
    ref = parity.normal_reference(crop.depth, p)       # sensitivity of the normal itself
    ok_o, ok_g = f.status == orc.OK, np.isfinite(k1)
    assert np.array_equal(ok_g, np.isfinite(k2)) and np.array_equal(ok_g, np.isfinite(n).all(-1))
    # validity agrees except where the singularity test of the regression is below resolution
    assert np.all(~np.isfinite(ref.sens[ok_o != ok_g]))
    assert np.all(k1[ok_g] == 0) and np.all(k2[ok_g] == 0)
    wp = ok_o & ok_g & (ref.sens <= 0.25 * parity.NORMAL_TOL)
    assert wp.sum() > 0.95 * ok_o.sum()
    assert parity.angle(n[wp], f.normal[wp]).max() <= parity.NORMAL_TOL
