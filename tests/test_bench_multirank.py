"""The N > 1 path of bench.py on CPU: world_size-2 gloo process groups.

Each rank solves its own copy of the workload (weak scaling, no data-path
collective); the only collective is the max over ranks of the step time.  The
reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, times, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.slowest_rank_ms(times[rank], dist)
    out[rank] = (ms, bench.job_value(ms, world, 4 * 65536))
    dist.destroy_process_group()


def test_slowest_rank_and_weak_scaling_value_gloo():
    import torch.multiprocessing as mp

    port = free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    times = [12.5, 17.25]
    mp.spawn(_worker, args=(2, port, times, out), nprocs=2, join=True)
    for r in range(2):
        ms, value = out[r]
        assert ms == 17.25
        assert value == pytest.approx(2 * 4 * 65536 / 17.25e-3)


def test_reference_arm_under_torchrun_prints_one_line_from_rank0():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--size", "1024",
           "--ref-sample", "4"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    res = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["unit"] == "eigvals/s" and rec["value"] > 0
