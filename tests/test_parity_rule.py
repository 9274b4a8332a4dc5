"""The comparison rule itself (oracle/parity.py), on hand-made fields: the
GPU parity tests are only as strong as this rule, so each way it could go
vacuous or wrong -- a pixel outside tolerance passing, an ill-posed pixel
gating, a validity flip away from the singularity threshold passing, k1 and
k2 swapped, NaN patterns that disagree -- is checked here on the CPU."""
import numpy as np

from oracle import BAD_NORMAL, OK, SINGULAR, Field, parity

PIVOT_TOL = 1e-5


def field(n=6):
    """n pixels, all valid and well away from the pivot threshold."""
    k1 = np.linspace(-3.0, 9.0, n)
    k2 = k1 - 2.0
    normal = np.tile([0.0, 0.6, 0.8], (n, 1))
    return Field(k1, k2, normal, np.full(n, OK), np.full(n, 0.3), np.zeros((n, 6)))


def ref_of(f, sens=None):
    return parity.Reference(f, np.zeros(f.k1.shape) if sens is None else np.asarray(sens, float), 0.0)


def test_tolerance_is_absolute_plus_relative():
    assert parity.tolerance(0.0) == 1e-4
    assert np.isclose(parity.tolerance(-50.0), 1e-4 + 5e-3)


def test_identical_output_passes():
    f = field()
    rep = parity.compare(f.k1, f.k2, f.normal, ref_of(f), PIVOT_TOL)
    assert rep.ok() and rep.n_well_posed == 6 and rep.max_rel_well_posed == 0.0
    assert rep.frac_within_tol_all == 1.0 and rep.max_normal_angle_well_posed < 1e-12


def test_error_just_inside_and_just_outside_tolerance():
    f = field()
    tol = parity.tolerance(f.k1[2])
    k1 = f.k1.copy()
    k1[2] += 0.99 * tol
    assert parity.compare(k1, f.k2, f.normal, ref_of(f), PIVOT_TOL).ok()
    k1[2] = f.k1[2] + 1.01 * tol
    rep = parity.compare(k1, f.k2, f.normal, ref_of(f), PIVOT_TOL)
    assert not rep.ok() and rep.n_well_posed_bad == 1 and rep.max_rel_well_posed > 1.0
    k2 = f.k2.copy()
    k2[4] -= 1.01 * parity.tolerance(f.k2[4])
    assert not parity.compare(f.k1, k2, f.normal, ref_of(f), PIVOT_TOL).ok()


def test_ill_posed_pixels_are_reported_not_gated():
    f = field()
    k1 = f.k1.copy()
    k1[1] += 10 * parity.tolerance(f.k1[1])
    sens = np.zeros(6)
    sens[1] = 0.3           # the oracle itself moves by 0.3 tolerances under rounding-sized noise
    rep = parity.compare(k1, f.k2, f.normal, ref_of(f, sens), PIVOT_TOL)
    assert rep.ok() and rep.n_well_posed == 5
    assert rep.frac_within_tol_all == 5 / 6
    sens[1] = 0.25          # at the limit the pixel is well-posed again and must agree
    assert not parity.compare(k1, f.k2, f.normal, ref_of(f, sens), PIVOT_TOL).ok()


def test_swapped_principal_curvatures_fail():
    f = field()
    assert not parity.compare(f.k2, f.k1, f.normal, ref_of(f), PIVOT_TOL).ok()


def test_validity_flip_far_from_the_threshold_fails():
    f = field()
    k1, k2, n = f.k1.copy(), f.k2.copy(), f.normal.copy()
    k1[3] = k2[3] = np.nan
    n[3] = np.nan
    rep = parity.compare(k1, k2, n, ref_of(f), PIVOT_TOL)
    assert not rep.ok() and rep.n_validity_mismatch == 1 and rep.n_validity_mismatch_band == 0
    # the oracle singular there instead, but with its smallest pivot far below the threshold
    g = field()
    g.status[3] = SINGULAR
    g.min_pivot[3] = PIVOT_TOL / 1e3
    g.k1[3] = g.k2[3] = np.nan
    rep = parity.compare(f.k1, f.k2, f.normal, ref_of(g), PIVOT_TOL)
    assert not rep.ok() and rep.n_validity_mismatch == 1


def test_validity_flip_at_the_threshold_is_allowed():
    g = field()
    f = field()
    g.status[3] = SINGULAR
    g.min_pivot[3] = 2 * PIVOT_TOL        # within the band of a factor 10 around the threshold
    g.k1[3] = g.k2[3] = np.nan
    rep = parity.compare(f.k1, f.k2, f.normal, ref_of(g), PIVOT_TOL)
    assert rep.ok() and rep.n_validity_mismatch_band == 1
    g.status[3] = BAD_NORMAL              # the 2x2 degeneracy test has no pivot record:
    assert not parity.compare(f.k1, f.k2, f.normal, ref_of(g), PIVOT_TOL).ok()   # not excused as such
    flips = np.zeros(6, bool)
    flips[3] = True                       # but excused where the probe flips the oracle's validity
    r = parity.Reference(g, np.zeros(6), 0.0, flips)
    rep = parity.compare(f.k1, f.k2, f.normal, r, PIVOT_TOL)
    assert rep.ok() and rep.n_validity_mismatch_band == 1
    flips[3], flips[2] = False, True      # a flip elsewhere excuses nothing
    assert not parity.compare(f.k1, f.k2, f.normal, r, PIVOT_TOL).ok()
    # a coarser implementation resolution widens the band
    g.status[3] = SINGULAR
    g.min_pivot[3] = 50 * PIVOT_TOL
    assert not parity.compare(f.k1, f.k2, f.normal, ref_of(g), PIVOT_TOL).ok()
    assert parity.compare(f.k1, f.k2, f.normal, ref_of(g), PIVOT_TOL, pivot_resolution=1e-4).ok()


def test_nan_pattern_must_agree_between_outputs():
    f = field()
    k2, n = f.k2.copy(), f.normal.copy()
    k2[0] = np.nan
    assert not parity.compare(f.k1, k2, f.normal, ref_of(f), PIVOT_TOL).ok()
    n[5, 1] = np.nan
    assert not parity.compare(f.k1, f.k2, n, ref_of(f), PIVOT_TOL).ok()


def test_normal_angle_is_reported():
    f = field()
    n = f.normal.copy()
    a = 3e-4
    n[2] = [0.0, 0.6 * np.cos(a) - 0.8 * np.sin(a), 0.6 * np.sin(a) + 0.8 * np.cos(a)]
    rep = parity.compare(f.k1, f.k2, n, ref_of(f), PIVOT_TOL)
    assert np.isclose(rep.max_normal_angle_well_posed, a, rtol=1e-6)


def test_normal_field_rule():
    n0 = np.tile([0.0, 0.0, 1.0], (4, 1))
    ref = parity.NormalReference(n0, np.full(4, OK), np.array([0.0, 0.0, 1e-3, np.inf]))
    good = n0.copy()
    assert parity.compare_normals(good, ref).ok()
    a = 2 * parity.NORMAL_TOL
    bad = n0.copy()
    bad[1] = [np.sin(a), 0.0, np.cos(a)]
    rep = parity.compare_normals(bad, ref)
    assert not rep.ok() and rep.n_well_posed_bad == 1 and np.isclose(rep.max_angle_well_posed, a)
    sensitive = n0.copy()
    sensitive[2] = [np.sin(a), 0.0, np.cos(a)]   # pixel 2 moved 1e-3 rad under the probe: not gated
    assert parity.compare_normals(sensitive, ref).ok()
    flip = n0.copy()
    flip[3] = np.nan                              # validity flips under the probe there: allowed
    assert parity.compare_normals(flip, ref).ok()
    flip[0] = np.nan                              # but not where it does not
    assert not parity.compare_normals(flip, ref).ok()


def test_condition_rule_and_excluded_pixels_are_reported():
    """The plainer rule (condition estimate <= 1e6) and the error on the pixels
    the probe excludes are reported, not gated."""
    f = field(10)
    f.cond = np.full(10, 10.0)
    f.cond[0] = 1e7                                  # ill-conditioned by the plainer rule
    sens = np.zeros(10)
    sens[[1, 2]] = 5.0                               # the probe excludes pixels 1 and 2
    k1 = f.k1.copy()
    k1[1] += 3.0 * parity.tolerance(f.k1[1])         # out of tolerance, excluded
    k1[2] += 0.5 * parity.tolerance(f.k1[2])
    k1[0] += 2.0 * parity.tolerance(f.k1[0])         # out of tolerance, not excluded
    rep = parity.compare(k1, f.k2, f.normal, parity.Reference(f, sens, 0.0), PIVOT_TOL)
    assert not rep.ok() and rep.n_well_posed_bad == 1
    assert rep.n_cond_well_posed == 9 and np.isclose(rep.frac_within_tol_cond, 8 / 9)
    assert rep.n_excluded == 2 and np.isclose(rep.max_rel_excluded, 3.0)
    assert 0.5 < rep.p999_rel_excluded <= 3.0
    assert rep.row()["excluded"] == 2 and np.isclose(rep.row()["cond_well_posed_frac"], 0.9)


def test_excluded_error_is_reported_against_the_probe_spread():
    f = field(4)
    sens = np.array([0.0, 2.0, 8.0, np.inf])      # pixel 3: the probe flips validity there
    k1 = f.k1.copy()
    k1[1] += 6.0 * parity.tolerance(f.k1[1])       # three times its spread
    k1[2] += 4.0 * parity.tolerance(f.k1[2])       # half its spread
    k1[3] += 100.0 * parity.tolerance(f.k1[3])     # no finite spread: not in the ratio
    rep = parity.compare(k1, f.k2, f.normal, parity.Reference(f, sens, 0.0), PIVOT_TOL)
    assert rep.ok() and rep.n_excluded == 3
    assert np.isclose(rep.max_excluded_over_spread, 3.0)
    assert 0.5 < rep.p99_excluded_over_spread <= 3.0
