"""The comparison rule between an implementation's per-pixel output and the
FP64 oracle.  TEST INFRASTRUCTURE (used by tests/, the smoke check and the
benchmark's reports only).

Tolerance: |dk| <= 1e-4 + 1e-4 |k| (1/m) for each principal curvature.

Which pixels the tolerance applies to.  The method runs a fixed number T of
re-weighted Gauss-Newton steps (Sec. 3.2.3).  Where those steps have settled,
the result depends on the data only; where they are still moving (noisy
windows, mixed surfaces), the iterate after T steps amplifies any
perturbation of the normal equations, and a single-precision implementation
perturbs them by its rounding.  So each pixel's sensitivity is measured on
the oracle itself: it is rerun with rounding-sized noise added to its normal
equations, to the sums of its initial-normal regression and to every
coordinate of p', for four seeds, and once with those sums formed in single
precision (the oracle's calibration mode, f32_sums).  A pixel whose answer
moves by more than a quarter of the tolerance in any of these runs is not
determined to that tolerance at single precision; every other pixel
("well-posed") must be within tolerance.

The size of the noise is calibrated, not assumed.  Summation error is bounded
by the sum of the magnitudes of the terms (u sum |t_i| per step), and by
Cauchy-Schwarz sum |w j_a j_c| <= sqrt(N_aa N_cc), sum |w eps j_a| <=
sqrt(N_aa E), E = sum w eps^2.  So the noise on entry (a, c) is a x
sqrt(N_aa N_cc) (x uniform in [-1, 1)): relative noise a on every entry of
the Jacobi-scaled matrix that the solve factorises, and likewise for the
right-hand side and the regression sums.  The oracle's single-precision mode
gives the error such sums actually make: its root mean square, in these
scaled units, is 0.17-0.19 sqrt(N) u for the normal matrix and 0.05-0.06
sqrt(N) u for the right-hand side (N window points, radii 3, 7, 11 of a
640 x 480 Kinect-like frame; 600 pixels x 5 iterations each), 0.21 sqrt(N) u
and 0.13 sqrt(N) u for the regression sums (N = 49).  The probe takes
a = PROBE_C sqrt(N) u with PROBE_C = 0.5, whose root mean square a / sqrt(3)
= 0.29 sqrt(N) u is 1.4-1.7 times the largest of these
(tests/test_oracle_probe.py measures it again).  Relative noise of 4 u on
each coordinate of p' stands for the rounding of single-precision
coordinates.  Relative noise on each entry (N u, the worst case of
recursive summation) is not a model of single precision: measured, the
relative error of near-zero entries reaches 10^5 u while the diagonal's stays
near sqrt(N) u.

Validity (NaN or not) must agree except where the oracle's own validity flips
in one of the probe's runs (which perturb the regression's degeneracy test
and every pivot alike), or where its smallest scaled pivot lies within a
factor `band` of the singularity threshold (or of `pivot_resolution`, the
smallest pivot the implementation's sums resolve, when that is larger).

The report also gives the statistics of the plainer rule that counts every
pixel valid in both as well-posed when the oracle's condition estimate (the
largest ratio of the largest to the smallest scaled Cholesky pivot of one
iteration) is at most 1e6, and the error on the pixels the probe excludes,
in tolerances and as a multiple of the spread of the oracle's own answers
under the probe at that pixel.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass

import numpy as np

from . import OK, SINGULAR, curvature_image, curvature_pixels

U = 2.0 ** -24
POINT_ULPS = 4        # relative rounding of a single-precision p' coordinate, in units of u
PROBE_C = 0.5         # probe amplitude a = PROBE_C sqrt(N) u (calibration above)
PROBE_SEEDS = (1, 2, 3, 4)
# The initial normal depends on five sums, so one probe run can leave it almost
# unmoved by chance (the angles of single runs on one pixel spread over a
# factor 10); sixteen runs give its largest response.  The full method's answer
# adds up hundreds of noise terms (42 entries per iteration and every
# coordinate), whose responses vary far less from run to run.
NORMAL_PROBE_SEEDS = tuple(range(1, 17))
COND_LIMIT = 1e6      # the plainer rule's condition threshold


def tolerance(k):
    return 1e-4 + 1e-4 * np.abs(k)


def window_points(p) -> int:
    s = max(int(p.stride), 1)
    n = 2 * (int(p.r) // s) + 1
    return n * n


def amplitude(npts: int) -> float:
    """the probe's noise amplitude for sums of npts terms"""
    return PROBE_C * float(np.sqrt(npts)) * U


@dataclass
class Reference:
    field: object            # oracle Field
    sens: np.ndarray         # sensitivity in units of the tolerance (inf: validity flips)
    amp: float
    flips: np.ndarray = None  # the oracle's validity changes in some probe run
    f32_within: float = float("nan")  # the oracle with its sums in single precision: fraction within tolerance


def reference(depth, p, nthreads=0, seeds=PROBE_SEEDS, uv=None) -> Reference:
    """Oracle output plus its sensitivity, for the whole image or the listed pixels."""
    run = (lambda q: curvature_image(depth, q, nthreads)) if uv is None else \
        (lambda q: curvature_pixels(depth, q, uv, nthreads))
    f = run(p)
    amp = amplitude(window_points(p))
    t1, t2 = tolerance(f.k1), tolerance(f.k2)
    sens = np.zeros_like(f.k1)
    flips = np.zeros(f.k1.shape, bool)
    f32_within = float("nan")
    probes = []
    for s in seeds:
        q = copy.copy(p)
        q.perturb, q.perturb_points, q.perturb_seed = amp, POINT_ULPS * U, s
        probes.append(q)
    q = copy.copy(p)
    q.f32_sums = 1          # sums formed in single precision
    probes.append(q)
    for q in probes:
        fp = run(q)
        with np.errstate(invalid="ignore"):
            d = np.maximum(np.abs(fp.k1 - f.k1) / t1, np.abs(fp.k2 - f.k2) / t2)
        flip = (fp.status == OK) != (f.status == OK)
        flips |= flip
        if q.f32_sums:
            both = (fp.status == OK) & (f.status == OK)
            f32_within = float(np.mean(d[both] <= 1)) if both.any() else 1.0
        d[flip & (f.status == OK)] = np.inf
        sens = np.maximum(sens, np.nan_to_num(d, nan=0.0))
    return Reference(f, sens, amp, flips, f32_within)


@dataclass
class Report:
    n_valid_oracle: int
    n_valid_both: int
    n_validity_mismatch: int          # not excused
    n_validity_mismatch_band: int     # excused: the oracle's validity flips under the probe, or at threshold
    n_well_posed: int
    n_well_posed_bad: int             # must be 0
    max_rel_well_posed: float         # max |dk| / tol over well-posed pixels
    frac_within_tol_all: float        # over all pixels valid in both
    max_normal_angle_well_posed: float
    nan_pattern_ok: bool              # k1, k2, normal NaN together
    n_cond_well_posed: int = 0        # valid in both with condition estimate <= COND_LIMIT
    frac_within_tol_cond: float = 1.0  # of those, within tolerance
    n_excluded: int = 0               # valid in both, not well-posed under the probe
    max_rel_excluded: float = 0.0     # max |dk| / tol over them
    p999_rel_excluded: float = 0.0    # 99.9th percentile of |dk| / tol over them
    p99_excluded_over_spread: float = 0.0   # |dk| over the probe's own spread (sens), 99th percentile
    max_excluded_over_spread: float = 0.0   # and maximum, over the excluded pixels with a finite spread
    frac_within_tol_f32_sums: float = float("nan")   # the oracle itself with single-precision sums

    def ok(self) -> bool:
        return self.n_validity_mismatch == 0 and self.n_well_posed_bad == 0 and self.nan_pattern_ok

    def summary(self) -> str:
        return (f"valid {self.n_valid_both}/{self.n_valid_oracle}, well-posed {self.n_well_posed} "
                f"({self.n_well_posed / max(self.n_valid_oracle, 1):.3f}), bad {self.n_well_posed_bad}, "
                f"max |dk|/tol {self.max_rel_well_posed:.3g}, all-pixel within tol "
                f"{self.frac_within_tol_all:.4f}, validity mismatches {self.n_validity_mismatch} "
                f"(+{self.n_validity_mismatch_band} excused), max normal angle "
                f"{self.max_normal_angle_well_posed:.3g} rad; cond<=1e6: {self.n_cond_well_posed} "
                f"({self.n_cond_well_posed / max(self.n_valid_oracle, 1):.3f}) of which within tol "
                f"{self.frac_within_tol_cond:.4f}; excluded {self.n_excluded}: max |dk|/tol "
                f"{self.max_rel_excluded:.3g}, p99.9 {self.p999_rel_excluded:.3g}; over the probe's spread "
                f"p99 {self.p99_excluded_over_spread:.3g}, max {self.max_excluded_over_spread:.3g}; "
                f"the oracle with single-precision sums within tol {self.frac_within_tol_f32_sums:.4f}")

    def row(self) -> dict:
        """the figures of one parity case, for the committed summary"""
        n = max(self.n_valid_oracle, 1)
        return {"valid_both": self.n_valid_both, "valid_oracle": self.n_valid_oracle,
                "well_posed_frac": self.n_well_posed / n, "bad": self.n_well_posed_bad,
                "worst_well_posed": self.max_rel_well_posed, "all_within": self.frac_within_tol_all,
                "validity_mismatch": self.n_validity_mismatch, "validity_excused": self.n_validity_mismatch_band,
                "cond_well_posed_frac": self.n_cond_well_posed / n, "cond_within": self.frac_within_tol_cond,
                "excluded": self.n_excluded, "max_excluded": self.max_rel_excluded,
                "p999_excluded": self.p999_rel_excluded, "p99_excluded_over_spread": self.p99_excluded_over_spread,
                "max_excluded_over_spread": self.max_excluded_over_spread,
                "f32_sums_within": self.frac_within_tol_f32_sums,
                "normal_angle": self.max_normal_angle_well_posed}


def compare(k1, k2, normal, ref: Reference, pivot_tol: float, band: float = 10.0,
            pivot_resolution: float = 0.0) -> Report:
    f = ref.field
    k1, k2 = np.asarray(k1, np.float64), np.asarray(k2, np.float64)
    g_valid = np.isfinite(k1)
    nan_ok = bool(np.array_equal(g_valid, np.isfinite(k2)))
    if normal is not None:
        normal = np.asarray(normal, np.float64)
        nan_ok = nan_ok and bool(np.array_equal(g_valid, np.isfinite(normal).all(-1)))
    o_valid = f.status == OK
    near = ((f.status == OK) | (f.status == SINGULAR)) & (f.min_pivot >= pivot_tol / band) & \
           (f.min_pivot <= max(pivot_tol, pivot_resolution) * band)
    if ref.flips is not None:
        near |= ref.flips
    mism = o_valid != g_valid
    both = o_valid & g_valid
    with np.errstate(invalid="ignore"):
        rel = np.maximum(np.abs(k1 - f.k1) / tolerance(f.k1), np.abs(k2 - f.k2) / tolerance(f.k2))
    wp = both & (ref.sens <= 0.25)
    ex = both & ~wp
    cond = f.cond if getattr(f, "cond", None) is not None else np.ones(f.k1.shape)
    cw = both & (cond <= COND_LIMIT)
    ang = np.zeros(0)
    if normal is not None and wp.any():
        c = np.clip(np.sum(normal[wp] * f.normal[wp], -1) /
                    (np.linalg.norm(normal[wp], axis=-1) * np.linalg.norm(f.normal[wp], axis=-1)), -1, 1)
        ang = np.arccos(c)
    # the excluded pixels' error against the spread of the oracle's own answers
    # under the probe (in tolerances); a validity flip has no finite spread
    fs = ex & np.isfinite(ref.sens)
    spread = rel[fs] / ref.sens[fs] if fs.any() else np.zeros(0)
    return Report(int(o_valid.sum()), int(both.sum()), int(np.sum(mism & ~near)), int(np.sum(mism & near)),
                  int(wp.sum()), int(np.sum(rel[wp] > 1)), float(rel[wp].max()) if wp.any() else 0.0,
                  float(np.mean(rel[both] <= 1)) if both.any() else 1.0,
                  float(ang.max()) if ang.size else 0.0, nan_ok,
                  int(cw.sum()), float(np.mean(rel[cw] <= 1)) if cw.any() else 1.0,
                  int(ex.sum()), float(rel[ex].max()) if ex.any() else 0.0,
                  float(np.quantile(rel[ex], 0.999)) if ex.any() else 0.0,
                  float(np.quantile(spread, 0.99)) if spread.size else 0.0,
                  float(spread.max()) if spread.size else 0.0, ref.f32_within)


# ---- the initial-normal field on its own (Sec. 3.2.1) --------------------------

NORMAL_TOL = 1e-4   # rad: angle between an implementation's normal and the oracle's


def angle(a, b):
    """angle (rad) between unit-ish normal fields a, b (... x 3); NaN where either is NaN"""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    c = np.sum(a * b, -1) / (np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1))
    s = np.linalg.norm(np.cross(a, b), axis=-1) / (np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1))
    return np.arctan2(s, c)


@dataclass
class NormalReference:
    normal: np.ndarray   # oracle normals, H x W x 3 (NaN unless status OK)
    status: np.ndarray
    sens: np.ndarray     # largest angle (rad) the perturbed runs moved it; inf where validity flips


def normal_reference(depth, p, seeds=NORMAL_PROBE_SEEDS, nthreads=0) -> NormalReference:
    """Oracle initial normals plus their sensitivity: the largest angle by
    which the probe's runs (noise of amplitude PROBE_C sqrt(N) u on the
    regression sums, N the patch points, and of 4 u on the coordinates of
    each patch point relative to the centre pixel's, as for the full method)
    and the single-precision sums move each normal; inf where validity flips."""
    from . import initial_normal_image
    n0, st = initial_normal_image(depth, p, nthreads)
    npts = (2 * int(p.rn) + 1) ** 2
    sens = np.zeros(st.shape)
    probes = []
    for seed in seeds:
        q = copy.copy(p)
        q.perturb, q.perturb_points, q.perturb_seed = amplitude(npts), POINT_ULPS * U, seed
        probes.append(q)
    q = copy.copy(p)
    q.f32_sums = 1
    probes.append(q)
    for q in probes:
        n1, st1 = initial_normal_image(depth, q, nthreads)
        flip = (st1 == OK) != (st == OK)
        both = (st1 == OK) & (st == OK)
        a = np.zeros(st.shape)
        a[both] = angle(n0[both], n1[both])
        a[flip] = np.inf
        sens = np.maximum(sens, a)
    return NormalReference(n0, st, sens)


@dataclass
class NormalReport:
    n_valid_oracle: int
    n_validity_mismatch: int          # outside the sensitive set
    n_validity_mismatch_sensitive: int
    n_well_posed: int
    n_well_posed_bad: int
    max_angle_well_posed: float

    def ok(self) -> bool:
        return self.n_validity_mismatch == 0 and self.n_well_posed_bad == 0

    def summary(self) -> str:
        return (f"valid {self.n_valid_oracle}, well-posed {self.n_well_posed}, bad {self.n_well_posed_bad}, "
                f"max angle {self.max_angle_well_posed:.3g} rad, validity mismatches "
                f"{self.n_validity_mismatch} (+{self.n_validity_mismatch_sensitive} sensitive)")


def compare_normals(normal, ref: NormalReference, tol: float = NORMAL_TOL) -> NormalReport:
    """Every well-posed pixel (valid in both, oracle moved by <= tol / 4 under
    the perturbations) within tol rad; validity agrees wherever the
    perturbations do not flip it."""
    g = np.asarray(normal, np.float64)
    g_valid = np.isfinite(g).all(-1)
    o_valid = ref.status == OK
    mism = g_valid != o_valid
    sensitive = ~np.isfinite(ref.sens)
    wp = g_valid & o_valid & (ref.sens <= 0.25 * tol)
    ang = angle(g[wp], ref.normal[wp]) if wp.any() else np.zeros(0)
    return NormalReport(int(o_valid.sum()), int((mism & ~sensitive).sum()), int((mism & sensitive).sum()),
                        int(wp.sum()), int((ang > tol).sum()), float(ang.max()) if ang.size else 0.0)
