"""The replicas' host-side coordination in bench.py (one process per GPU
under torchrun), run as two gloo ranks on the CPU: the barrier, the maximum
of the timed durations over the ranks, the whole-job rate, and the reference
arm, which runs and prints on rank 0 only."""
import contextlib
import io
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.Ranks(world, "cpu")
    r.barrier()
    slowest = r.max_over_ranks(1.5 + rank)          # rank 1 "took" 2.5 s
    rate = bench.whole_job_rate(world, 1000, slowest)
    buf = io.StringIO()
    args = bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-seconds", "1"])
    with contextlib.redirect_stdout(buf):
        ret = bench.run_reference(args, rank, world)
    r.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "rate": rate, "ret": ret, "printed": buf.getvalue()}, f)


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(worker, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == 2.5                     # the same maximum on every rank
        assert r["rate"] == pytest.approx(2 * 1000 / 2.5)
        assert r["ret"] is None
    assert res[1]["printed"] == ""                     # other ranks exit without work
    lines = [l for l in res[0]["printed"].splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["ms_per_step"] > 0


def test_single_rank_needs_no_process_group():
    import bench
    r = bench.Ranks(1, "cpu")
    r.barrier()
    assert r.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_rate(1, 10, 2.0) == 5.0
