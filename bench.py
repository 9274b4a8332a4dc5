"""Throughput of dense per-pixel principal curvature on synthetic Kinect-like
range images: 640 x 480, window radius 7 (15 x 15), 5 re-weighted iterations,
FP32 (the per-pixel quadric fit of Spek, Li, Drummond, arXiv 1707.00385).

One step = the whole method (back-projection, initial normal, 5 iterations,
eigen step, refined normal) over a batch of FRAMES distinct frame buffers
(about 157 MB of ranges, more than the 129 MB L2, so no step reads another's
inputs from L2), enqueued as one pc_compute_batch call (a CUDA graph: frame
table copy, queue reset, one persistent kernel over all tiles).

Prints one JSON line.  `value` is Mpixel/s over the device-timed region with
inputs resident in HBM; `per_frame_launches` is the same with one pc_compute
launch per frame; `uneven_batch` runs 64 frames of mixed resolutions
(320x240, 512x424 time-of-flight, 640x480, 1280x720) in one batch call
against 64 plain launches, `small_frames` 512 frames of 64x48 likewise; `e2e` is the metric through pc_compute_host_batch
with pinned host buffers (host-to-device ranges and device-to-host k1, k2,
normals inside the timed region, pipelined in chunks against the compute;
`one_call_per_frame` is pc_compute_host once per frame); `outputs` times
the organised point cloud (pc_backproject, against the HBM peak) and the
initial-normal field (pc_initial_normals); `roofline` reports the persistent
kernel against the FP32 ALU peak; `cpu_baseline` times the FP64 oracle on a
bounded sample on the host, and the same leg's FP64 answers on one frame are
what `precision` measures the precision variants against (rank 0, one GPU).

--impl reference times the oracle alone, on the host cores, on the same
workload (each step a bounded sample).

Multi-GPU (torchrun): every rank runs the same per-rank workload on its own
GPU (replicas; the method needs no exchange), timing is bracketed by barriers
and the max over ranks is reported (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W, RADIUS, ITERS = 480, 640, 7, 5
FRAMES = 128          # frame buffers per step
SCENES = 8            # distinct seeded scenes (seeds 0..7), repeated over the buffers
FLOP_PER_VISIT = 101  # counted FP32 operations per window point per iteration
FLOP_PER_SOLVE = 250  # per pixel per iteration (6x6 system, update)
FLOP_PER_NORMAL_PT = 12
FP32_LANES_PER_SM = 128
SERVE_REQUESTS = 20000       # the serving workload's trace (Poisson arrivals at 2000/s)
SERVE_HALF_REQUESTS = 4000   # the trace offered at half the measured batched capacity
SERVE_VERIFY = 100           # served requests whose results are checked after the timed traces
# batches the continuous-batching server keeps on the GPU.  GB300, 3000 requests: 2 / 3 / 4 in
# flight served 1403 / 1406 / 1390 frames/s at 2000/s offered, p99 6.57 / 5.91 / 5.56 ms at half
# capacity (one launch per frame: 5.8-6.5 ms across the same runs)
SERVE_INFLIGHT = 3
METRIC = ("Mpixel/s of (k1,k2) at 640x480 r=7 vs FP32 roofline; "
          "served frames/s + p99 at <=1e-3 rel err")
WORKLOAD = "640x480 Kinect-like synthetic scenes, window radius 7 (15x15), 5 IRLS iterations, FP32"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=FRAMES)
    ap.add_argument("--scenes", type=int, default=SCENES)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests of the serving trace (default 20000)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-inflight", type=int, default=SERVE_INFLIGHT,
                    help="batches the continuous-batching server keeps on the GPU at once")
    ap.add_argument("--fp32-peak-seconds", type=float, default=1.0,
                    help="timed length of each form of the multiply-add microbenchmark")
    ap.add_argument("--report", choices=["serve", "accuracy", "outputs", "table2", "sweep",
                                         "tensorcore", "fp32peak"],
                    default=None,
                    help="instead of the benchmark line: serve = the "
                         "serving trace and a point at half capacity; accuracy = error against "
                         "analytic ground truth; outputs = the organised outputs alone; table2 = the "
                         "paper's timing grid (3 resolutions x 9x9, 21x21, sparse 37x37 windows); sweep = "
                         "throughput and FP32-roofline fraction for window radii 1..12 at 640x480; "
                         "tensorcore = the window moments on the FP32 pipe against tensor cores; "
                         "fp32peak = the multiply-add microbenchmark alone")
    return ap.parse_args(argv)


def scenes(n):
    import synth
    return [synth.kinect_scene(seed) for seed in range(n)]


UNEVEN_SIZES = [(240, 320, "kinect"), (424, 512, "tof"), (480, 640, "kinect"), (720, 1280, "kinect")]


# Small frames: the size of the smallest parity case, cut from the seeded scenes.
SMALL_H, SMALL_W = 48, 64
SMALL_FRAMES = 512
SMALL_DISTINCT = 16


def synth_crop(scene, v0, u0, h, w):
    import synth
    return synth.crop(scene, v0, u0, h, w)


def uneven_scenes(per_size=2):
    """Seeded frames of the four resolutions (seeds 1000+), per_size of each."""
    import synth
    out = []
    for j, (h, w, noise) in enumerate(UNEVEN_SIZES):
        for i in range(per_size):
            out.append(synth.kinect_scene(1000 + 10 * j + i, H=h, W=w, noise=noise))
    return out


def counted_flop(depth, r=RADIUS, T=ITERS, rn=3):
    """Counted FP32 work of one frame: for every pixel with a valid range and
    enough valid neighbours, T * (101 |W_p| + 250) + 12 |N_p|, where |W_p| and
    |N_p| are the valid points of its (2r+1)^2 window and (2rn+1)^2 patch."""
    valid = (depth > 0) & np.isfinite(depth)
    v = valid.astype(np.int64)

    def box(rad):
        c = np.pad(v, ((1, 0), (1, 0))).cumsum(0).cumsum(1)
        Hh, Ww = v.shape
        y0 = np.clip(np.arange(Hh) - rad, 0, Hh)
        y1 = np.clip(np.arange(Hh) + rad + 1, 0, Hh)
        x0 = np.clip(np.arange(Ww) - rad, 0, Ww)
        x1 = np.clip(np.arange(Ww) + rad + 1, 0, Ww)
        return c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0]

    nw, nn = box(r), box(rn)
    use = valid & (nw >= 6) & (nn >= 3)
    return float(np.sum(np.where(use, T * (FLOP_PER_VISIT * nw + FLOP_PER_SOLVE) + FLOP_PER_NORMAL_PT * nn, 0)))


def measured_hbm_gbs():
    """HBM copy bandwidth measured on this GPU model (MEASURED_PEAKS.json), or None"""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def cpu_model():
    """CPU model name of the host (lscpu, else /proc/cpuinfo), for the baseline's record"""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for l in out.splitlines():
            if l.lower().startswith("model name"):
                return l.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for l in open("/proc/cpuinfo"):
            if l.lower().startswith(("model name", "cpu model")):
                return l.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def alu_peak_tflops(sms, sm_mhz):
    """FP32 issue ceiling derived from the SM count and a clock: 128 FP32 lanes
    per SM, 2 FLOP per fused multiply-add"""
    return sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def fp32_peak(pc, dev, stream, index, seconds=1.0):
    """The measured FP32 ceiling: the library's multiply-add microbenchmark
    (pc_fp32_peak_kernel, packed FP32x2 and scalar) timed with CUDA events on
    its stream over about `seconds`, SM clocks sampled meanwhile."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    blocks, iters = props.multi_processor_count * 4, 8192
    sink = torch.empty(blocks * 256, device=dev)
    out = {"kernel": "pc_fp32_peak_kernel: 32 independent fused multiply-add chains per thread, "
                     f"{blocks} CTAs of 256 threads, {iters} rounds"}
    h = stream.cuda_stream
    for packed in (1, 0):
        st, flop = pc.pc_fp32_peak_kernel(blocks, iters, packed, sink.data_ptr(), sink.numel(), h)
        if st != pc.PC_OK:
            raise RuntimeError(f"pc_fp32_peak_kernel: status {st}")
        for _ in range(20):
            pc.pc_fp32_peak_kernel(blocks, iters, packed, sink.data_ptr(), sink.numel(), h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n = max(20, int(seconds / max(flop / 75e12, 1e-6)))
        clk = Clocks(index)
        clk.__enter__()
        e0.record(stream)
        for _ in range(n):
            pc.pc_fp32_peak_kernel(blocks, iters, packed, sink.data_ptr(), sink.numel(), h)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.__exit__(None, None, None)
        c = clk.summary()
        tf = flop * n / (e0.elapsed_time(e1) * 1e-3) / 1e12
        key = "packed_fp32x2" if packed else "scalar"
        out[key] = {"tflops": tf, "sm_mhz": c["sm_mhz"], "reasons": c["reasons"],
                    "derived_peak_at_that_clock": alu_peak_tflops(props.multi_processor_count, c["sm_mhz"])
                    if c["sm_mhz"] else None}
    out["tflops"] = max(out["packed_fp32x2"]["tflops"], out["scalar"]["tflops"])
    return out


def kernel_sources_hash():
    """hash of the code of the files that define the fused kernels (device
    code and the structures it reads), without comments and blank space:
    host-only files and comment edits do not change the kernel"""
    import re
    d = os.path.join(ROOT, "paper_1707_00385_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if (f.startswith("pc_fit") and f.endswith((".cu", ".cuh"))) or f in ("pc_f32x2.cuh", "pc_internal.h"):
            code = open(os.path.join(d, f)).read()
            code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
            code = re.sub(r"//[^\n]*", " ", code)
            h.update(f.encode())
            h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(frames):
    """DRAM bytes of one persistent launch over `frames` 640x480 frames, from
    the committed ncu record of the full-size launch (128 frames), if it was
    taken on the current kernel sources.  Larger launches scale in proportion
    (their results overflow L2 the same way); smaller ones keep results in L2
    and are not reported."""
    p = os.path.join(ROOT, "profiles", "k_fit_r7_640x480_traffic.txt")
    if not os.path.exists(p):
        return None
    kv = dict(l.strip().split("=", 1) for l in open(p) if "=" in l and not l.startswith("#"))
    if kv.get("kernel_sources_sha256_16") != kernel_sources_hash():
        return None
    base = int(kv["frames_per_launch"])
    if frames < base:
        return None
    return float(kv["dram_bytes_per_launch"]) * frames / base


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(frames_np, intr, seconds):
    """The FP64 oracle as it stands on the host cores, on rows of the first
    frame(s) until about `seconds` of work: Mpixel/s."""
    import oracle
    p = oracle.params(*intr, r=RADIUS, T=ITERS)
    cores = oracle.max_threads()
    done, t0 = 0, time.perf_counter()
    rows = 8
    fi, v0 = 0, 0
    while time.perf_counter() - t0 < seconds and fi < len(frames_np):
        d = frames_np[fi]
        vv, uu = np.mgrid[v0:min(v0 + rows, H), 0:W]
        uv = np.stack([uu.ravel(), vv.ravel()], 1)
        oracle.curvature_pixels(d, p, uv, nthreads=cores)
        done += uv.shape[0]
        v0 += rows
        if v0 >= H:
            fi, v0 = fi + 1, 0
    dt = time.perf_counter() - t0
    return {"value": done / dt / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"{done} pixels ({done // W} rows of 640x480 seeded scenes), "
                      f"FP64 C oracle, {dt:.1f} s"}


class Ranks:
    """Host-side coordination of the replicas (one process per GPU, torchrun):
    a barrier around each timed region and the maximum of a duration over the
    ranks.  The method needs no data exchange; these are the only collectives.
    `device` is where the reduction buffer lives (the rank's GPU under NCCL,
    the CPU under gloo)."""

    def __init__(self, world, device):
        self.world, self.device = world, device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(self, x):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(world, units_per_rank, seconds):
    """Aggregate throughput of the replicas: every rank processed units_per_rank
    units; the job took the slowest rank's time (weak scaling)."""
    return float(world) * units_per_rank / seconds


def run_reference(args, rank, world):
    if rank != 0:
        return
    frames = [s.depth for s in scenes(1)]
    intr = (525.0, 525.0, 319.5, 239.5)
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(frames, intr, seconds=max(2.0, args.cpu_seconds / 4))
        if i >= args.warmup:
            vals.append(cb)
    v = statistics.median(c["value"] for c in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Mpixel/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            # the time one step of the device arm's workload (args.frames frames) would take at this rate
            "ms_per_step": args.frames * H * W / (v * 1e6) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "bounded row bands of frame 0 per step",
                       "ms_per_step": f"extrapolated to {args.frames} frames of {W}x{H} from the sample's rate"},
            "cpu_baseline": {"value": v, "unit": "Mpixel/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "cpu_model": vals[0]["cpu_model"], "nproc": vals[0]["nproc"],
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def serve_trace(scenes_, n, rate, seed, batched=True, plain=True, inflight=SERVE_INFLIGHT, verify=0):
    """Serves n requests arriving as a Poisson process at `rate` per second,
    each a frame drawn uniformly from scenes_ (host, page-locked), with the
    continuous-batching server and with one launch per frame; then, when
    verify > 0, checks the results of `verify` more served requests."""
    import torch
    from paper_1707_00385_gb300.serve import (GpuExecutor, PlainExecutor, Request, Server, device_budget,
                                              poisson_arrivals)
    pool = [(torch.from_numpy(s.depth).pin_memory(), s.intrinsics) for s in scenes_]
    rng = np.random.default_rng(seed)
    t = poisson_arrivals(n, rate, seed)
    pick = rng.integers(0, len(pool), n)
    budget = device_budget(0.5)
    out = {"requests": n, "offered_per_s": rate, "resolutions": [f"{w}x{h}" for h, w, _ in UNEVEN_SIZES],
           "budget_bytes": budget}
    modes = ([("continuous_batching", GpuExecutor, dict(max_batch_frames=64, inflight=inflight))]
             if batched else []) + \
            ([("one_launch_per_frame", PlainExecutor, dict(max_batch_frames=1, inflight=64))] if plain else [])
    # untimed start-up: a trace of the same rate (another seed) first, which
    # also fills the executor's pool of page-locked result buffers
    nw = min(n, 2000)
    tw = poisson_arrivals(nw, rate, seed + 1000)
    pick_w = np.random.default_rng(seed + 1000).integers(0, len(pool), nw)
    for name, Ex, kw in modes:
        ex = Ex(RADIUS, ITERS, slots=kw["inflight"]) if Ex is GpuExecutor else Ex(RADIUS, ITERS)
        warm = [Request(-1 - i, *pool[pick_w[i]], float(tw[i])) for i in range(nw)]
        Server(ex, budget, **kw).run(warm)
        reqs = [Request(i, *pool[pick[i]], float(t[i])) for i in range(n)]
        st = Server(ex, budget, **kw).run(reqs)
        ex.close()
        out[name] = {"frames_per_s": st.frames_per_s, "mpixel_per_s": st.mpixel_per_s, "p50_ms": st.p50_ms,
                     "p99_ms": st.p99_ms, "mean_batch": st.mean_batch, "batches": st.batches,
                     "peak_device_bytes": st.peak_device_bytes}
    if batched and verify:
        out["served_results"] = served_results_check(pool, rate, seed + 2000, verify, inflight)
    return out


def served_results_check(pool, rate, seed, n, inflight):
    """Untimed: n requests of the same mix served by the continuous-batching
    server with their results kept, each compared with its frame computed
    alone by pc_compute (the path the parity tests check against the FP64
    oracle).  Equal bits mean the served answers carry exactly that path's
    error against the oracle (the `precision` key)."""
    import torch
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300.serve import GpuExecutor, Request, Server, device_budget, poisson_arrivals
    alone = []
    for d, intr in pool:
        c = pc.Curvature(*intr, window_radius=RADIUS, iterations=ITERS)
        alone.append([x.cpu().numpy() for x in c(d.cuda())])
        c.close()
    t = poisson_arrivals(n, rate, seed)
    pick = np.random.default_rng(seed).integers(0, len(pool), n)
    ex = GpuExecutor(RADIUS, ITERS, slots=inflight, keep_results=True)
    reqs = [Request(i, *pool[pick[i]], float(t[i])) for i in range(n)]
    st = Server(ex, device_budget(0.5), max_batch_frames=64, inflight=inflight).run(reqs)
    ex.close()
    equal = all(r.error is None and all(np.array_equal(x.numpy(), y, equal_nan=True)
                                        for x, y in zip((r.k1, r.k2, r.normal), alone[pick[r.rid]]))
                for r in reqs)
    return {"requests": n, "mean_batch": st.mean_batch, "equal_to_frame_alone": bool(equal)}


def _interior(mask, r):
    """pixels whose whole (2r+1)^2 window lies inside mask (edges and corners
    excluded, as the paper's evaluation removes them)"""
    m = mask.astype(np.int64)
    c = np.pad(m, ((1, 0), (1, 0))).cumsum(0).cumsum(1)
    Hh, Ww = m.shape
    y0, y1 = np.clip(np.arange(Hh) - r, 0, Hh), np.clip(np.arange(Hh) + r + 1, 0, Hh)
    x0, x1 = np.clip(np.arange(Ww) - r, 0, Ww), np.clip(np.arange(Ww) + r + 1, 0, Ww)
    box = c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0]
    return mask & (box == (2 * r + 1) ** 2)


def accuracy_report(args):
    """Accuracy of the method itself against analytic ground truth (GPU path):
    the synthetic rows of the paper's Table 1 (sphere 10 cm, cylinder 9 cm,
    torus 10/3 cm), curvature error against depth noise on a 100 mm sphere,
    and the angular error of the refined normal against the initial one."""
    import torch
    import synth
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300 import build as pcbuild
    pcbuild.build()
    cam = synth.kinect_camera(480, 640)
    wall = synth.Plane(np.array([0.0, 0.0, 1.0]), 1.5)

    def run(scene, r, T=5, **kw):
        c = pc.Curvature(*scene.intrinsics, window_radius=r, iterations=T, **kw)
        k1, k2, n = c(torch.from_numpy(scene.depth).cuda())
        torch.cuda.synchronize()
        c.close()
        return k1.cpu().numpy(), k2.cpu().numpy(), n.cpu().numpy()

    objects = {
        "sphere_10cm": synth.Sphere(np.array([0.0, 0.0, 0.8]), 0.10),
        "cylinder_9cm": synth.Cylinder(np.array([0.0, 0.0, 0.8]), np.array([0.0, 1.0, 0.0]), 0.09, 0.4),
        "torus_10_3cm": synth.Torus(np.array([0.0, 0.0, 0.8]), np.array([0.0, -0.6, -0.8]), 0.10, 0.03),
    }
    windows = [("r7_dense", 7, 1), ("37x37_stride3", 18, 3)]
    for noise_name, noise in (("none", None), ("kinect", synth.kinect_noise)):
        for name, obj in objects.items():
            sc = synth.render(cam, [obj, wall], noise=noise, rng=np.random.default_rng(1))
            for wname, r, st in windows:
                k1, k2, _ = run(sc, r, stride=st)
                m = _interior(sc.label == 0, r) & np.isfinite(k1)
                e = np.concatenate([(k1 - sc.gt_k1)[m], (k2 - sc.gt_k2)[m]]) / 1000.0   # mm^-1
                print(json.dumps({"table1_row": name, "noise": noise_name, "window": wname, "pixels": int(m.sum()),
                                  "expected_k_per_mm": [float(np.nanmean(sc.gt_k1[m]) / 1000), float(np.nanmean(sc.gt_k2[m]) / 1000)],
                                  "computed_k_per_mm": [float(np.mean(k1[m]) / 1000), float(np.mean(k2[m]) / 1000)],
                                  "rms_per_mm": float(np.sqrt(np.mean(e * e))), "sigma_per_mm": float(np.std(e))}),
                      flush=True)
    sph = objects["sphere_10cm"]
    for sigma_mm in (0.0, 0.5, 1.0, 2.0, 3.0, 4.0, 5.0):
        sc = synth.render(cam, [sph, wall], noise=synth.const_noise(sigma_mm * 1e-3) if sigma_mm else None,
                          rng=np.random.default_rng(2))
        row = {"noise_mm": sigma_mm}
        for tag, kw in (("ours", {}), ("ours_rejection", {"reject": 1})):
            k1, k2, n = run(sc, 7, **kw)
            m = _interior(sc.label == 0, 7) & np.isfinite(k1)
            e = np.concatenate([(k1 - 10.0)[m], (k2 - 10.0)[m]])
            row[tag + "_rms_per_m"] = float(np.sqrt(np.mean(e * e)))
            if tag == "ours":
                ang = np.degrees(np.arccos(np.clip(np.sum(n[m] * sc.gt_normal[m], -1), -1, 1)))
                row["refined_normal_mean_deg"] = float(np.mean(ang))
        _, _, n0 = run(sc, 7, T=0)
        m = _interior(sc.label == 0, 7) & np.isfinite(n0[..., 0])
        ang0 = np.degrees(np.arccos(np.clip(np.sum(n0[m] * sc.gt_normal[m], -1), -1, 1)))
        row["initial_normal_mean_deg"] = float(np.mean(ang0))
        print(json.dumps({"sphere_100mm_vs_noise": row}), flush=True)


BIG_SIDE = 4096   # the organised outputs' roofline case: 16.8 Mpixel, 268 MB of HBM traffic > L2


def outputs_report(curv, depth, stream, device_time, steps, sm_mhz):
    """Organised outputs of the same frames: pc_backproject (HBM-bound: 4 B in,
    12 B out per pixel) and pc_initial_normals, per 640x480 frame (one launch
    each, launch-latency bound) and on one 4096 x 4096 image tiled from the
    frames (the kernels' own throughput; inputs and outputs larger than L2)."""
    import torch
    H_, W_ = depth[0].shape
    F_ = len(depth)
    xyz = [torch.empty((H_, W_, 3), device=depth[0].device) for _ in range(F_)]
    n0 = [torch.empty((H_, W_, 3), device=depth[0].device) for _ in range(F_)]
    ms_bp = device_time(lambda: [curv.backproject(depth[i], xyz[i], stream=stream) for i in range(F_)], steps) / steps / F_
    ms_n0 = device_time(lambda: [curv.initial_normals(depth[i], n0[i], stream=stream) for i in range(F_)],
                        steps) / steps / F_
    del xyz, n0
    reps = (BIG_SIDE + H_ - 1) // H_, (BIG_SIDE + W_ - 1) // W_
    big = torch.cat([torch.cat([depth[(i * reps[1] + j) % F_] for j in range(reps[1])], 1)
                     for i in range(reps[0])], 0)[:BIG_SIDE, :BIG_SIDE].contiguous()
    bxyz = torch.empty((BIG_SIDE, BIG_SIDE, 3), device=big.device)
    bn0 = torch.empty((BIG_SIDE, BIG_SIDE, 3), device=big.device)
    big_steps = 4 * steps
    ms_bbp = device_time(lambda: curv.backproject(big, bxyz, stream=stream), big_steps) / big_steps
    ms_bn0 = device_time(lambda: curv.initial_normals(big, bn0, stream=stream), big_steps) / big_steps
    del big, bxyz, bn0
    px = BIG_SIDE * BIG_SIDE
    hbm_peak = measured_hbm_gbs()
    gbs = 16 * px / (ms_bbp * 1e-3) / 1e9
    normal_flop = px * (FLOP_PER_NORMAL_PT * 49 + 20)     # 7x7 patch, 2x2 solve and normalisation
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    alu_peak = alu_peak_tflops(props.multi_processor_count, sm_mhz) if sm_mhz else None
    achieved_n0 = normal_flop / (ms_bn0 * 1e-3) / 1e12
    return {
        "backproject": {
            "ms_per_640x480_frame": ms_bp, "ms_4096x4096": ms_bbp, "mpixel_per_s_4096x4096": px / ms_bbp / 1e3,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak if hbm_peak else None, "algorithmic_bytes_per_pixel": 16,
                         "case": "one 4096x4096 image", "peak_basis": "measured HBM copy bandwidth"}},
        "initial_normals": {
            "ms_per_640x480_frame": ms_n0, "ms_4096x4096": ms_bn0, "mpixel_per_s_4096x4096": px / ms_bn0 / 1e3,
            "roofline": {"bound": "alu", "achieved": achieved_n0, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": achieved_n0 / alu_peak if alu_peak else None,
                         "counted_flop_per_pixel": FLOP_PER_NORMAL_PT * 49 + 20, "case": "one 4096x4096 image",
                         "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                       f"{sm_mhz or 0:.0f} MHz sampled SM clock (derived)"}},
    }


# The precision variants the error columns cover: (name, context parameters,
# 16-bit storage format); their pivot thresholds are PRECISION_PIVOTS.
PRECISION_VARIANTS = [("fp32", {}, 0), ("fp32_kahan", {"kahan": 1}, 0),
                      ("fp32_fp64solve", {"pivot_tol": 1e-7, "fp64_solve_cond": 1e6}, 0),
                      ("fp16_storage", {}, 1), ("bf16_storage", {}, 2)]
PRECISION_PIVOTS = (1e-5, 1e-7)


def oracle_answers(depth, intr, radii, pivots=PRECISION_PIVOTS):
    """Part of the cpu_baseline leg (rank 0, one GPU, host cores): the FP64
    oracle's answers on one frame, which the precision columns measure the
    GPU variants against.  Returns {(r, pivot): (k1, k2, valid)} as plain arrays."""
    import oracle
    out = {}
    for r in radii:
        for piv in pivots:
            f = oracle.curvature_image(depth, oracle.params(*intr, r=r, T=ITERS, pivot_tol=piv))
            out[(r, piv)] = (f.k1, f.k2, f.status == oracle.OK)
    return out


def precision_rows(radii, refs, echo=False):
    """Error of each precision variant on frame 0 of the seeded scenes against
    refs = oracle_answers(frame 0, its intrinsics, radii), with its time per
    frame: one row per variant and window radius."""
    import torch
    import paper_1707_00385_gb300 as pc
    s = scenes(1)[0]
    intr = s.intrinsics
    d = torch.from_numpy(s.depth).cuda()
    rows = []
    for r in radii:
        for name, kw, fmt in PRECISION_VARIANTS:
            fk1, fk2, ok = refs[(r, kw.get("pivot_tol", 1e-5))]
            c = pc.Curvature(*intr, window_radius=r, iterations=ITERS, **kw)
            if fmt:
                packed, base = c.pack(d, fmt)
                run = lambda: c.compute_packed(packed, base, fmt)
            else:
                run = lambda: c(d)
            for _ in range(3):
                out = run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                out = run()
            e1.record()
            torch.cuda.synchronize()
            k1, k2 = out[0].cpu().numpy(), out[1].cpu().numpy()
            c.close()
            both = ok & np.isfinite(k1)
            err = np.maximum(np.abs(k1 - fk1), np.abs(k2 - fk2))[both]
            rel = np.maximum(np.abs(k1 - fk1) / (1e-4 + 1e-4 * np.abs(fk1)),
                             np.abs(k2 - fk2) / (1e-4 + 1e-4 * np.abs(fk2)))[both]
            # relative error with a floor of 1 m^-1 (flat surfaces have k near 0)
            relk = np.maximum(np.abs(k1 - fk1) / np.maximum(np.abs(fk1), 1.0),
                              np.abs(k2 - fk2) / np.maximum(np.abs(fk2), 1.0))[both]
            rows.append({"variant": name, "window_radius": r, "ms_per_frame": e0.elapsed_time(e1) / 10,
                         "valid_both": int(both.sum()), "validity_mismatch": int(np.sum(ok != np.isfinite(k1))),
                         "median_abs_dk": float(np.median(err)), "p99_abs_dk": float(np.quantile(err, 0.99)),
                         "frac_within_tol": float(np.mean(rel <= 1)),
                         "frac_rel_err_le_1e-3": float(np.mean(relk <= 1e-3))})
            if echo:
                print(json.dumps(rows[-1]), flush=True)
    return rows


# The paper's timing grid (Table 2): image sizes and patches; the 37 x 37 patch is
# "sparsely sampled" without a stride, read here as every third pixel (radius 18).
TABLE2_SIZES = [(480, 640), (424, 512), (240, 320)]
TABLE2_WINDOWS = [("9x9", 4, 1), ("21x21", 10, 1), ("37x37 sparse (stride 3)", 18, 3)]


def table2_report(args):
    """Time per frame of the whole method on the paper's Table 2 grid, one
    pc_compute launch per frame (as a per-frame timing) and batches of 32
    frames (pc_compute_batch), T = 5 iterations (the paper states none)."""
    import torch
    import synth
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300 import build as pcbuild
    pcbuild.build()
    rows = []
    stream = torch.cuda.Stream()
    for H, W in TABLE2_SIZES:
        sc = [synth.kinect_scene(2000 + i, H=H, W=W, noise="tof" if (H, W) == (424, 512) else "kinect")
              for i in range(4)]
        frames = 32
        depth = [torch.from_numpy(sc[i % 4].depth).cuda() for i in range(frames)]
        outs = [(torch.empty((H, W), device="cuda"), torch.empty((H, W), device="cuda"),
                 torch.empty((H, W, 3), device="cuda")) for _ in range(frames)]
        for name, r, stride in TABLE2_WINDOWS:
            c = pc.Curvature(*sc[0].intrinsics, window_radius=r, iterations=ITERS, stride=stride)
            args_b = [(depth[i], sc[i % 4].intrinsics) + outs[i] for i in range(frames)]

            def per_frame():
                for i in range(frames):
                    c(depth[i], *outs[i], stream=stream)

            def batched():
                c.batch(args_b, stream=stream)

            res = {"size": f"{W}x{H}", "window": name, "window_radius": r, "stride": stride, "iterations": ITERS}
            for key, fn in (("per_frame_ms", per_frame), ("batched_ms_per_frame", batched)):
                with torch.cuda.stream(stream):
                    for _ in range(3):
                        fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                reps = 5
                with torch.cuda.stream(stream):
                    for _ in range(reps):
                        fn()
                e1.record(stream)
                torch.cuda.synchronize()
                res[key] = e0.elapsed_time(e1) / (reps * frames)
            res["mpixel_per_s_batched"] = H * W / res["batched_ms_per_frame"] / 1e3
            c.close()
            rows.append(res)
            print(json.dumps(res), flush=True)
    return rows


def sweep_report(args):
    """Throughput and counted-FLOP fraction of the FP32 peak for dense window
    radii 1..12 (the unrolled kernels), 640 x 480 frames, T = 5, one batch of
    32 frame buffers per step (the headline's launch form at a quarter of its
    size), CUDA events over 5 steps after 3 warm-up ones."""
    import torch
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300 import build as pcbuild
    pcbuild.build()
    sc = scenes(8)
    intr = sc[0].intrinsics
    F = 32
    depth = [torch.from_numpy(sc[i % 8].depth).cuda() for i in range(F)]
    outs = [(torch.empty((H, W), device="cuda"), torch.empty((H, W), device="cuda"),
             torch.empty((H, W, 3), device="cuda")) for _ in range(F)]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    stream = torch.cuda.Stream()
    rows = []
    for r in range(1, 13):
        c = pc.Curvature(*intr, window_radius=r, iterations=ITERS)
        frames = [(depth[i], intr) + outs[i] for i in range(F)]
        flop = sum(counted_flop(sc[i % 8].depth, r=r) for i in range(F))
        with torch.cuda.stream(stream):
            for _ in range(3):
                c.batch(frames, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = Clocks(0)
        clk.__enter__()
        e0.record(stream)
        reps = 0
        while reps < 5 or time.perf_counter() - t0 < 0.6:   # long enough for several clock samples
            if reps == 0:
                t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                c.batch(frames, stream=stream)
            reps += 1
            if reps % 5 == 0:
                stream.synchronize()
        e1.record(stream)
        torch.cuda.synchronize()
        clk.__exit__(None, None, None)
        mhz = clk.summary()["sm_mhz"]
        ms = e0.elapsed_time(e1) / reps
        c.close()
        res = {"window_radius": r, "window": f"{2 * r + 1}x{2 * r + 1}", "ms_per_frame": ms / F,
               "mpixel_per_s": F * H * W / ms / 1e3, "counted_tflop_per_s": flop / ms / 1e9, "sm_mhz": mhz,
               "frac_fp32_peak": flop / ms / 1e-3 / (alu_peak_tflops(sms, mhz) * 1e12) if mhz else None}
        rows.append(res)
        print(json.dumps(res), flush=True)
    return rows


def api_overhead(pc, curv, dev, stream, calls=300):
    """Host time of one call of the C ABI (argument checks, tile plan, launch),
    without the device work it enqueues: pc_compute on one 8 x 32 frame and
    pc_compute_batch on that frame alone, each call made with the stream idle
    (synchronised before it) and timed on the host; median over `calls`
    calls, through ctypes with the pointers prepared beforehand."""
    import torch
    d = torch.ones((8, 32), device=dev)
    k1, k2, n = torch.empty_like(d), torch.empty_like(d), torch.empty((8, 32, 3), device=dev)
    h = stream.cuda_stream
    fr = (pc.pc_frame * 1)()
    fr[0] = pc.pc_frame(d.data_ptr(), 8, 32, 525.0, 525.0, 16.0, 4.0, k1.data_ptr(), k2.data_ptr(), n.data_ptr())
    calls_of = {
        "pc_compute_us": lambda: pc.pc_compute(curv.ctx, d.data_ptr(), 8, 32, h, k1.data_ptr(), k2.data_ptr(),
                                               n.data_ptr()),
        "pc_compute_batch_us": lambda: pc.pc_compute_batch(curv.ctx, fr, 1, h),
    }
    out = {"frame": "8x32, r = 7, T = 5", "calls": calls, "timing": "median host time of one call, stream idle"}
    for name, call in calls_of.items():
        for _ in range(20):
            call()
        ts = []
        for _ in range(calls):
            stream.synchronize()
            t0 = time.perf_counter()
            call()
            ts.append(time.perf_counter() - t0)
        stream.synchronize()
        out[name] = statistics.median(ts) * 1e6
    return out


def tensorcore_report(args):
    """The window moments of one 640 x 480 frame's 5 iterations (307,200
    windows of 15 x 15) on the FP32 pipe and on tensor cores
    (pc_moments_probe), CUDA events over 20 launches after 3 warm-up ones, SM
    clocks sampled; beside it the whole curvature kernel per frame."""
    import torch
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300 import build as pcbuild
    pcbuild.build()
    props = torch.cuda.get_device_properties(0)
    sink = torch.empty(512 * props.multi_processor_count, device="cuda")
    stream = torch.cuda.Stream()
    h = stream.cuda_stream
    pixels = H * W
    res = {"pixels": pixels, "iterations": ITERS, "window": "15x15"}
    for mode, name in ((0, "fp32_pipe"), (1, "tensor_cores_3xtf32")):
        st, blocks = pc.pc_moments_probe(mode, pixels, ITERS, sink.data_ptr(), sink.numel(), h)
        if st != pc.PC_OK:
            raise RuntimeError(f"pc_moments_probe mode {mode}: status {st}")
        for _ in range(3):
            pc.pc_moments_probe(mode, pixels, ITERS, sink.data_ptr(), sink.numel(), h)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clk = Clocks(0)
        clk.__enter__()
        e0.record(stream)
        reps = 20
        for _ in range(reps):
            pc.pc_moments_probe(mode, pixels, ITERS, sink.data_ptr(), sink.numel(), h)
        e1.record(stream)
        torch.cuda.synchronize()
        clk.__exit__(None, None, None)
        res[name] = {"ms_per_frame": e0.elapsed_time(e1) / reps, "ctas": blocks, "sm_mhz": clk.summary()["sm_mhz"]}
    res["tensor_over_fp32"] = res["tensor_cores_3xtf32"]["ms_per_frame"] / res["fp32_pipe"]["ms_per_frame"]
    # the whole method, one persistent launch over 32 frames
    sc = scenes(8)
    F = 32
    depth = [torch.from_numpy(sc[i % 8].depth).cuda() for i in range(F)]
    outs = [(torch.empty((H, W), device="cuda"), torch.empty((H, W), device="cuda"),
             torch.empty((H, W, 3), device="cuda")) for _ in range(F)]
    c = pc.Curvature(*sc[0].intrinsics, window_radius=RADIUS, iterations=ITERS)
    frames = [(depth[i], sc[i % 8].intrinsics) + outs[i] for i in range(F)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            c.batch(frames, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(5):
            c.batch(frames, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    c.close()
    res["whole_method_ms_per_frame"] = e0.elapsed_time(e1) / (5 * F)
    print(json.dumps({"tensorcore": res}), flush=True)
    return res


def main():
    args = parse()
    if args.report == "fp32peak":
        import torch
        import paper_1707_00385_gb300 as pc
        from paper_1707_00385_gb300 import build as pcbuild
        pcbuild.build()
        res = fp32_peak(pc, torch.device("cuda", 0), torch.cuda.Stream(), 0, seconds=max(args.fp32_peak_seconds, 1.0))
        print(json.dumps({"fp32peak": res}), flush=True)
        return
    if args.report == "tensorcore":
        tensorcore_report(args)
        return
    if args.report == "sweep":
        sweep_report(args)
        return
    if args.report == "table2":
        table2_report(args)
        return
    if args.report == "accuracy":
        accuracy_report(args)
        return
    if args.report == "outputs":
        import torch
        import paper_1707_00385_gb300 as pc
        from paper_1707_00385_gb300 import build as pcbuild
        pcbuild.build()
        sc = scenes(max(1, min(args.scenes, args.frames)))
        depth = [torch.from_numpy(sc[i % len(sc)].depth).cuda() for i in range(args.frames)]
        curv = pc.Curvature(*sc[0].intrinsics, window_radius=RADIUS, iterations=ITERS)
        stream = torch.cuda.Stream()

        def device_time(step, steps):
            with torch.cuda.stream(stream):
                for _ in range(max(3, args.warmup)):
                    step()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)

        clk = Clocks(0)
        clk.__enter__()
        out = outputs_report(curv, depth, stream, device_time, max(2, args.steps // 4), None)
        clk.__exit__(None, None, None)
        mhz = clk.summary()["sm_mhz"]
        if mhz:   # the ceiling at the clock sampled while the kernels ran
            rf = out["initial_normals"]["roofline"]
            rf["peak"] = alu_peak_tflops(torch.cuda.get_device_properties(0).multi_processor_count, mhz)
            rf["frac"] = rf["achieved"] / rf["peak"]
            rf["peak_basis"] = rf["peak_basis"].replace(" 0 MHz", f" {mhz:.0f} MHz")
        print(json.dumps({"outputs": out, "sm_mhz": mhz}), flush=True)
        curv.close()
        return
    if args.report == "serve":
        # the serving workload: 20,000 requests at 2,000/s, then a point at half the
        # measured batched capacity
        un = uneven_scenes(2)
        n = args.serve_requests if args.serve_requests is not None else 20000
        full = serve_trace(un, n, args.serve_rate, seed=11, inflight=args.serve_inflight)
        print(json.dumps({"serve": full, "inflight": args.serve_inflight}), flush=True)
        cap = full["continuous_batching"]["frames_per_s"]
        half = serve_trace(un, n, 0.5 * cap, seed=12, inflight=args.serve_inflight)
        print(json.dumps({"serve_half_capacity": half}), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_1707_00385_gb300 as pc
    from paper_1707_00385_gb300 import build as pcbuild
    pcbuild.build()

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    barrier = Ranks(world, dev).barrier
    max_over_ranks = Ranks(world, dev).max_over_ranks

    nsc = max(1, min(args.scenes, args.frames))
    sc = scenes(nsc)
    intr = sc[0].intrinsics
    F = args.frames
    host = [sc[i % nsc].depth for i in range(F)]
    flop_frame = [counted_flop(s.depth) for s in sc]
    flop_step = sum(flop_frame[i % nsc] for i in range(F))
    depth = [torch.from_numpy(h).to(dev) for h in host]          # F distinct buffers
    k1 = [torch.empty((H, W), device=dev) for _ in range(F)]
    k2 = [torch.empty((H, W), device=dev) for _ in range(F)]
    nrm = [torch.empty((H, W, 3), device=dev) for _ in range(F)]
    curv = pc.Curvature(*intr, window_radius=RADIUS, iterations=ITERS)
    stream = torch.cuda.Stream(device=dev)
    batch_args = [(depth[i], intr, k1[i], k2[i], nrm[i]) for i in range(F)]

    def step_batch():
        curv.batch(batch_args, stream=stream)

    def step_frames():
        for i in range(F):
            curv(depth[i], k1[i], k2[i], nrm[i], stream=stream)

    def device_time(step, steps, clocks=None):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctxm = Clocks(local) if clocks is not None else None
        if ctxm:
            ctxm.__enter__()
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if ctxm:
            ctxm.__exit__(None, None, None)
            clocks.update(ctxm.summary())
        barrier()
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1))

    # ---- device-timed region: inputs resident in HBM, one batch call per step
    clocks = {}
    ms = device_time(step_batch, args.steps, clocks)
    ms_step = ms / args.steps
    value = whole_job_rate(world, args.steps * F * H * W, ms / 1e3) / 1e6
    launch_ms = ms_step   # one persistent kernel per step
    # the same frames, one pc_compute launch per frame
    ms_pf = device_time(step_frames, max(2, args.steps // 2))
    pf_value = whole_job_rate(world, max(2, args.steps // 2) * F * H * W, ms_pf / 1e3) / 1e6

    # ---- uneven frames (four resolutions): one batch call vs plain launches
    un = uneven_scenes(2)
    un_dev = []
    for i in range(64):
        s_ = un[i % len(un)]
        d_ = torch.from_numpy(s_.depth).to(dev)
        un_dev.append((d_, s_.intrinsics, torch.empty_like(d_), torch.empty_like(d_),
                       torch.empty(d_.shape + (3,), device=dev)))
    un_px = sum(a[0].numel() for a in un_dev)
    un_ctx = [pc.Curvature(*s_.intrinsics, window_radius=RADIUS, iterations=ITERS) for s_ in un]

    def step_un_batch():
        curv.batch(un_dev, stream=stream)

    def step_un_frames():
        for i, (d_, _, a_, b_, n_) in enumerate(un_dev):
            un_ctx[i % len(un)](d_, a_, b_, n_, stream=stream)

    ub_steps = max(2, args.steps // 4)
    ms_ub = device_time(step_un_batch, ub_steps)
    ms_uf = device_time(step_un_frames, ub_steps)
    uneven = {"frames": 64, "resolutions": [f"{w}x{h}" for h, w, _ in UNEVEN_SIZES],
              "distinct_scenes": len(un), "pixels": un_px,
              "batch_frames_per_s": whole_job_rate(world, 64 * ub_steps, ms_ub / 1e3),
              "plain_launch_frames_per_s": whole_job_rate(world, 64 * ub_steps, ms_uf / 1e3),
              "batch_ms": ms_ub / ub_steps, "plain_ms": ms_uf / ub_steps}
    for c_ in un_ctx:
        c_.close()

    # ---- small frames (64x48, the size of the smallest parity case): 512 in one
    # batch call vs one launch each, where one frame fills only 12 of 152 SMs
    sm_scenes = [synth_crop(sc[i % nsc], 20 + 25 * i, 30 + 35 * i, SMALL_H, SMALL_W) for i in range(SMALL_DISTINCT)]
    sm_dev = []
    for i in range(SMALL_FRAMES):
        s_ = sm_scenes[i % SMALL_DISTINCT]
        d_ = torch.from_numpy(s_.depth).to(dev)
        sm_dev.append((d_, s_.intrinsics, torch.empty_like(d_), torch.empty_like(d_),
                       torch.empty(d_.shape + (3,), device=dev)))
    sm_ctx = [pc.Curvature(*s_.intrinsics, window_radius=RADIUS, iterations=ITERS) for s_ in sm_scenes]

    def step_sm_batch():
        curv.batch(sm_dev, stream=stream)

    def step_sm_frames():
        for i, (d_, _, a_, b_, n_) in enumerate(sm_dev):
            sm_ctx[i % SMALL_DISTINCT](d_, a_, b_, n_, stream=stream)

    ms_sb = device_time(step_sm_batch, ub_steps)
    ms_sf = device_time(step_sm_frames, ub_steps)
    small = {"frames": SMALL_FRAMES, "size": f"{SMALL_W}x{SMALL_H}", "distinct_crops": SMALL_DISTINCT,
             "inputs": "L2-resident (12 KB per frame)",
             "batch_frames_per_s": whole_job_rate(world, SMALL_FRAMES * ub_steps, ms_sb / 1e3),
             "plain_launch_frames_per_s": whole_job_rate(world, SMALL_FRAMES * ub_steps, ms_sf / 1e3),
             "batch_ms": ms_sb / ub_steps, "plain_ms": ms_sf / ub_steps}
    for c_ in sm_ctx:
        c_.close()

    # ---- serving: Poisson arrivals of the mixed-resolution frames, continuous
    # batching vs one launch per frame (same frames, same trace): the stated
    # 20,000-request trace, then a shorter one offered at half the batched capacity
    serve_res = serve_trace(un, args.serve_requests if args.serve_requests is not None else SERVE_REQUESTS,
                            args.serve_rate, seed=11, inflight=args.serve_inflight, verify=SERVE_VERIFY)
    half_rate = 0.5 * serve_res["continuous_batching"]["frames_per_s"]
    half_n = SERVE_HALF_REQUESTS if args.serve_requests is None else max(1, args.serve_requests // 5)
    serve_res["half_capacity"] = serve_trace(un, half_n, half_rate, seed=12, inflight=args.serve_inflight)
    serve_res["inflight_batches"] = args.serve_inflight

    # ---- end to end through the host-memory entry point (pinned buffers)
    hd = [torch.from_numpy(h).pin_memory() for h in host]
    hk1 = [torch.empty((H, W)).pin_memory() for _ in range(F)]
    hk2 = [torch.empty((H, W)).pin_memory() for _ in range(F)]
    hn = [torch.empty((H, W, 3)).pin_memory() for _ in range(F)]
    e2e_ctx = pc.Curvature(*intr, window_radius=RADIUS, iterations=ITERS)
    host_frames = [(hd[i], intr, hk1[i], hk2[i], hn[i]) for i in range(F)]

    def step_host_batch():
        # pipelined: chunks of frames copied in, computed and copied out on overlapping streams
        e2e_ctx.host_batch(host_frames, stream=stream)
        stream.synchronize()

    def step_host_frames():
        for i in range(F):
            e2e_ctx.compute_host(hd[i], hk1[i], hk2[i], hn[i], stream=stream)
        stream.synchronize()

    def wall_time(step, steps):
        for _ in range(max(1, args.warmup)):
            step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        t1 = time.perf_counter()
        barrier()
        return max_over_ranks(t1 - t0)

    e2e_steps = max(2, args.steps // 2)
    e2e_s = wall_time(step_host_batch, e2e_steps)
    e2e_val = whole_job_rate(world, e2e_steps * F * H * W, e2e_s) / 1e6
    # host path and batched device path give the same numbers
    step_batch()
    torch.cuda.synchronize()
    same = bool(np.array_equal(hk1[0].numpy(), k1[0].cpu().numpy(), equal_nan=True))
    e2e_pf_steps = max(1, args.steps // 4)
    e2e_pf_val = whole_job_rate(world, e2e_pf_steps * F * H * W, wall_time(step_host_frames, e2e_pf_steps)) / 1e6

    # ---- organised outputs (point cloud, initial-normal field)
    outputs = outputs_report(curv, depth, stream, device_time, max(2, args.steps // 4), clocks.get("sm_mhz"))

    # ---- host cost of one API call (what a per-frame caller pays beside the kernel)
    overhead = api_overhead(pc, curv, dev, stream)

    # ---- cpu_baseline leg (rank 0, one GPU): the FP64 oracle timed on the host
    # cores, and its answers on frame 0 for the precision columns (radius 7)
    cpu_leg = rank == 0 and world == 1 and not args.no_cpu_baseline
    precision = None
    if cpu_leg:
        cpu_line = cpu_baseline([s.depth for s in sc], intr, args.cpu_seconds)
        s0 = scenes(1)[0]
        precision = precision_rows((RADIUS,), oracle_answers(s0.depth, s0.intrinsics, (RADIUS,)))

    # ---- roofline of the persistent kernel: counted FP32 work vs the FP32 ALU
    # ceiling, derived at the SM clock sampled during the timed region and
    # measured by the multiply-add microbenchmark
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = clocks.get("sm_mhz")
    peak = alu_peak_tflops(props.multi_processor_count, sm_mhz) if sm_mhz else None
    measured = fp32_peak(pc, dev, stream, local, seconds=args.fp32_peak_seconds)
    achieved = flop_step / (launch_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak if peak else None,
            "traffic": recorded_traffic(F),
            "kernel": f"k_fit_batch<7> (fused normal + IRLS + eigen), one persistent launch over {F} 640x480 frames",
            "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                          f"{sm_mhz or 0:.0f} MHz, the median SM clock sampled during the timed region (derived)",
            "measured_fp32_peak": measured, "frac_of_measured": achieved / measured["tflops"],
            "launch_ms": launch_ms, "counted_flop_per_launch": flop_step}

    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "window_radius": RADIUS, "iterations": ITERS,
                       "frames_per_step": F, "distinct_scenes": nsc,
                       "l2": (f"inputs larger than L2: {F} distinct frame buffers "
                              f"({F * H * W * 4 / 1e6:.0f} MB of ranges) per step"
                              if F * H * W * 4 > 129e6 else
                              f"inputs smaller than L2 ({F * H * W * 4 / 1e6:.0f} MB): profiling case only"),
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_val, "unit": "Mpixel/s", "h2d_bytes_per_step": F * H * W * 4,
                    "d2h_bytes_per_step": F * H * W * 4 * 5, "api": "pc_compute_host_batch",
                    "matches_device_path": same,
                    "one_call_per_frame": {"api": "pc_compute_host", "value": e2e_pf_val, "unit": "Mpixel/s"}},
            "outputs": outputs,
            "per_frame_launches": {"value": pf_value, "unit": "Mpixel/s", "ms_per_frame": ms_pf / max(2, args.steps // 2) / F},
            "uneven_batch": uneven,
            "small_frames": small,
            "serve": serve_res,
            "precision": precision,
            "api_overhead": overhead,
            "gpu_launches": args.steps,
            "clocks": clocks,
            "roofline": roof}
    if cpu_leg:
        line["cpu_baseline"] = cpu_line
    if rank == 0:
        print(json.dumps(line), flush=True)
    curv.close()
    e2e_ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
