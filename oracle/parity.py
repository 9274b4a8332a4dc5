"""The comparison rule between an implementation's per-pixel output and the
FP64 oracle.  TEST INFRASTRUCTURE (used by tests/, the smoke check and the
benchmark's reports only).

Tolerance: |dk| <= 1e-4 + 1e-4 |k| (1/m) for each principal curvature.

Which pixels the tolerance applies to.  The method runs a fixed number T of
re-weighted Gauss-Newton steps (Sec. 3.2.3).  Where those steps have settled,
the result depends on the data only; where they are still moving (noisy
windows, mixed surfaces, near-singular systems), the iterate after T steps
amplifies any perturbation of the normal equations.  A single-precision
implementation perturbs them by its rounding, about N u relative for sums of
N window terms (u = 2^-24, the standard bound of recursive summation).  So
each pixel's sensitivity is measured on the oracle itself: it is rerun with
the entries of its normal equations and of its initial-normal regression
multiplied by 1 + a x (x uniform in [-1, 1), a = N u) and every coordinate
of every p' multiplied by 1 + 4 u x (the rounding of a single-precision
coordinate), for two seeds; a pixel whose answer moves by more than a quarter
of the tolerance is not determined to that tolerance at single precision.
Every other pixel ("well-posed") must be within tolerance.

Validity (NaN or not) must agree except where the oracle's smallest scaled
pivot lies within a factor `band` of the singularity threshold (or of
`pivot_resolution`, the smallest pivot the implementation's sums resolve,
when that is larger), where the decision itself is below the
implementation's resolution.
"""
from __future__ import annotations

import copy
from dataclasses import dataclass

import numpy as np

from . import OK, SINGULAR, BAD_NORMAL, curvature_image, curvature_pixels

U = 2.0 ** -24
POINT_ULPS = 4   # relative rounding of a single-precision p' coordinate, in units of u


def tolerance(k):
    return 1e-4 + 1e-4 * np.abs(k)


def window_points(p) -> int:
    s = max(int(p.stride), 1)
    n = 2 * (int(p.r) // s) + 1
    return n * n


@dataclass
class Reference:
    field: object            # oracle Field
    sens: np.ndarray         # sensitivity in units of the tolerance (inf: validity flips)
    amp: float


def reference(depth, p, nthreads=0, seeds=(1, 2), uv=None) -> Reference:
    """Oracle output plus its sensitivity, for the whole image or the listed pixels."""
    run = (lambda q: curvature_image(depth, q, nthreads)) if uv is None else \
        (lambda q: curvature_pixels(depth, q, uv, nthreads))
    f = run(p)
    amp = window_points(p) * U
    t1, t2 = tolerance(f.k1), tolerance(f.k2)
    sens = np.zeros_like(f.k1)
    for s in seeds:
        q = copy.copy(p)
        q.perturb, q.perturb_points, q.perturb_seed = amp, POINT_ULPS * U, s
        fp = run(q)
        with np.errstate(invalid="ignore"):
            d = np.maximum(np.abs(fp.k1 - f.k1) / t1, np.abs(fp.k2 - f.k2) / t2)
        d[np.isnan(d) & (f.status == OK)] = np.inf
        sens = np.maximum(sens, np.nan_to_num(d, nan=0.0))
    return Reference(f, sens, amp)


@dataclass
class Report:
    n_valid_oracle: int
    n_valid_both: int
    n_validity_mismatch: int          # outside the threshold band
    n_validity_mismatch_band: int     # inside the band (allowed)
    n_well_posed: int
    n_well_posed_bad: int             # must be 0
    max_rel_well_posed: float         # max |dk| / tol over well-posed pixels
    frac_within_tol_all: float        # over all pixels valid in both
    max_normal_angle_well_posed: float
    nan_pattern_ok: bool              # k1, k2, normal NaN together

    def ok(self) -> bool:
        return self.n_validity_mismatch == 0 and self.n_well_posed_bad == 0 and self.nan_pattern_ok

    def summary(self) -> str:
        return (f"valid {self.n_valid_both}/{self.n_valid_oracle}, well-posed {self.n_well_posed} "
                f"({self.n_well_posed / max(self.n_valid_oracle, 1):.3f}), bad {self.n_well_posed_bad}, "
                f"max |dk|/tol {self.max_rel_well_posed:.3g}, all-pixel within tol "
                f"{self.frac_within_tol_all:.4f}, validity mismatches {self.n_validity_mismatch} "
                f"(+{self.n_validity_mismatch_band} at threshold), max normal angle "
                f"{self.max_normal_angle_well_posed:.3g} rad")


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
    near |= f.status == BAD_NORMAL  # the 2x2 degeneracy test has no pivot record; counted as band
    mism = o_valid != g_valid
    both = o_valid & g_valid
    with np.errstate(invalid="ignore"):
        rel = np.maximum(np.abs(k1 - f.k1) / tolerance(f.k1), np.abs(k2 - f.k2) / tolerance(f.k2))
    wp = both & (ref.sens <= 0.25)
    ang = np.zeros(0)
    if normal is not None and wp.any():
        c = np.clip(np.sum(normal[wp] * f.normal[wp], -1) /
                    (np.linalg.norm(normal[wp], axis=-1) * np.linalg.norm(f.normal[wp], axis=-1)), -1, 1)
        ang = np.arccos(c)
    return Report(int(o_valid.sum()), int(both.sum()), int(np.sum(mism & ~near)), int(np.sum(mism & near)),
                  int(wp.sum()), int(np.sum(rel[wp] > 1)), float(rel[wp].max()) if wp.any() else 0.0,
                  float(np.mean(rel[both] <= 1)) if both.any() else 1.0,
                  float(ang.max()) if ang.size else 0.0, nan_ok)


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


def normal_reference(depth, p, seeds=(1, 2), nthreads=0) -> NormalReference:
    """Oracle initial normals plus their sensitivity to relative perturbations
    of the regression sums of size a = N u (N the patch points), as for the
    full method."""
    from . import initial_normal_image
    n0, st = initial_normal_image(depth, p, nthreads)
    npts = (2 * int(p.rn) + 1) ** 2
    sens = np.zeros(st.shape)
    for seed in seeds:
        q = copy.copy(p)
        q.perturb = npts * U
        q.perturb_seed = seed
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
