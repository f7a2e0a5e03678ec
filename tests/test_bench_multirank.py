"""Multi-rank logic of bench.py on the CPU (gloo, world size 2).

Under torchrun every rank advances its own replica of the workload; the
benchmark takes the slowest rank's time and reports the whole job's
throughput.  The reference arm runs on rank 0 only; the other ranks exit
without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    mine = [0.5, 2.0][rank]
    slowest = bench.max_over_ranks(dist, mine, "cpu")
    value = bench.job_mlups(world, 256 ** 3, 100, slowest)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"slowest": slowest, "value": value}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_job_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["slowest"] == 2.0
        assert r["value"] == pytest.approx(2 * 256 ** 3 * 100 / 2.0 / 1e6)


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(None, 1.25, "cpu") == 1.25
    assert bench.job_mlups(1, 1000, 10, 1e-3) == pytest.approx(10.0)


def _run_reference(rank, world):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                           "--gpus", str(world), "--steps", "2", "--warmup", "3", "--size", "64"],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_only_on_rank_zero():
    other = _run_reference(1, 2)
    assert other.returncode == 0, other.stderr
    assert other.stdout.strip() == ""
    first = _run_reference(0, 2)
    assert first.returncode == 0, first.stderr
    lines = [l for l in first.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["n_gpus"] == 2 and d["steps"] == 2 and d["warmup"] == 3
    assert d["metric"] == bench.METRIC and d["unit"] == "MLUPs/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
