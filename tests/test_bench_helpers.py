"""Host-side pieces of bench.py that feed the reported numbers: the counted
work behind the roofline fraction (against a brute-force count), the
recorded DRAM traffic (reported only for the kernel sources it was taken on,
scaled by frames), the clock summary parsed from nvidia-smi lines, and the
whole-job rate."""
import numpy as np
import pytest

import bench


def brute_counted_flop(depth, r, T, rn):
    H, W = depth.shape
    valid = (depth > 0) & np.isfinite(depth)
    total = 0.0
    for v in range(H):
        for u in range(W):
            if not valid[v, u]:
                continue
            nw = valid[max(0, v - r):v + r + 1, max(0, u - r):u + r + 1].sum()
            nn = valid[max(0, v - rn):v + rn + 1, max(0, u - rn):u + rn + 1].sum()
            if nw >= 6 and nn >= 3:
                total += T * (bench.FLOP_PER_VISIT * nw + bench.FLOP_PER_SOLVE) + bench.FLOP_PER_NORMAL_PT * nn
    return total


@pytest.mark.parametrize("r,T", [(7, 5), (3, 3), (1, 1)])
def test_counted_flop_matches_brute_force(r, T):
    rng = np.random.default_rng(r)
    d = rng.uniform(0.5, 3.0, (23, 37)).astype(np.float32)
    d[rng.random(d.shape) < 0.3] = 0.0
    d[4, 5], d[6, 7] = np.nan, np.inf
    assert bench.counted_flop(d, r=r, T=T) == brute_counted_flop(d, r, T, 3)


def test_counted_flop_of_one_isolated_window():
    """a single valid 15 x 15 block inside invalid surroundings: only its
    centre sees the whole window and patch"""
    d = np.zeros((31, 31), np.float32)
    d[8:23, 8:23] = 1.0
    full = bench.counted_flop(d, r=7, T=5)
    d2 = d.copy()
    d2[15, 15] = 0.0      # drop the centre: its own work goes, and one point from every other window
    assert full - bench.counted_flop(d2, r=7, T=5) > 5 * (bench.FLOP_PER_VISIT * 225 + bench.FLOP_PER_SOLVE)


def test_recorded_traffic_follows_the_kernel_sources(monkeypatch):
    rec = bench.os.path.join(bench.ROOT, "profiles", "k_fit_r7_640x480_traffic.txt")
    kv = dict(l.strip().split("=", 1) for l in open(rec) if "=" in l and not l.startswith("#"))
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: kv["kernel_sources_sha256_16"])
    base = bench.recorded_traffic(128)
    assert base == float(kv["dram_bytes_per_launch"]) > 0
    assert bench.recorded_traffic(256) == pytest.approx(2 * base)
    assert bench.recorded_traffic(64) is None               # results of a small launch stay in L2
    monkeypatch.setattr(bench, "kernel_sources_hash", lambda: "0000000000000000")
    assert bench.recorded_traffic(128) is None              # counters of other kernel code are not reported


def test_kernel_hash_ignores_comments_only(tmp_path, monkeypatch):
    import shutil
    src = tmp_path / "paper_1707_00385_gb300" / "csrc"
    shutil.copytree(bench.os.path.join(bench.ROOT, "paper_1707_00385_gb300", "csrc"), src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_sources_hash()
    f = src / "pc_fit.cuh"
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n  ", 3))
    assert bench.kernel_sources_hash() == h0
    f.write_text(text.replace("TILE_W", "TILE_W ", 1) + "\nstatic int extra_symbol;\n")
    assert bench.kernel_sources_hash() != h0


def test_clock_summary():
    c = bench.Clocks(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines = []
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_whole_job_rate_is_weak_scaling():
    assert bench.whole_job_rate(1, 1000, 2.0) == 500.0
    assert bench.whole_job_rate(4, 1000, 2.0) == 2000.0


def test_fp32_ceiling_is_derived_from_the_given_clock():
    import bench
    assert abs(bench.alu_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    assert abs(bench.alu_peak_tflops(152, 1477.0) / bench.alu_peak_tflops(152, 2070.0) - 1477 / 2070) < 1e-12


def test_cpu_model_is_named():
    import bench
    m = bench.cpu_model()
    assert isinstance(m, str) and m.strip()


def test_oracle_answers_keys_and_shapes(orc):
    """The cpu_baseline leg's FP64 answers for the precision columns: one
    (k1, k2, valid) triple per window radius and pivot threshold."""
    import synth
    s = synth.crop(synth.kinect_scene(3), 200, 300, 12, 20)
    refs = bench.oracle_answers(s.depth, s.intrinsics, (2, 3))
    assert set(refs) == {(r, p) for r in (2, 3) for p in bench.PRECISION_PIVOTS}
    for k1, k2, ok in refs.values():
        assert k1.shape == k2.shape == ok.shape == (12, 20) and ok.dtype == bool
        assert np.isfinite(k1[ok]).all() and np.all(k1[ok] >= k2[ok])
    assert {p.get("pivot_tol", 1e-5) for _, p, _ in bench.PRECISION_VARIANTS} <= set(bench.PRECISION_PIVOTS)
