"""The benchmark's host-side contract on the CPU: the reference arm's JSON
line, the multi-rank helpers over gloo with two ranks, and the reference arm
under torchrun (rank 0 alone prints)."""
import json
import os
import subprocess
import sys

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(cmd, env=None, timeout=300):
    e = dict(os.environ, **(env or {}))
    return subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=timeout, env=e)


def test_reference_arm_json_line():
    r = _run([sys.executable, "bench.py", "--impl", "reference", "--config", "C1", "--steps", "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1


def _helpers_worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(world)
    m = bench.reduce_max(float(rank + 1) * 1.5, world)
    out[rank] = m
    dist.destroy_process_group()


def test_multi_rank_helpers_over_gloo():
    world, port = 2, 29631
    out = mp.Manager().dict()
    mp.spawn(_helpers_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0] == out[1] == 3.0          # the maximum over ranks reaches every rank


def test_reference_arm_under_torchrun_two_ranks():
    r = _run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
              "--master-addr", "127.0.0.1", "--master-port", "29632", "bench.py", "--impl", "reference",
              "--config", "C1", "--steps", "1", "--warmup", "1"], env={"OMP_NUM_THREADS": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1                   # rank 0 alone prints
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
