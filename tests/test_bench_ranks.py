"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the
max-over-ranks timing, the whole-job throughput, and the reference arm
printing one JSON line from rank 0 under torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        v = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        out[rank] = v
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
        assert dict(out) == {0: 15.0, 1: 15.0}


def test_job_throughput_is_weak_scaling():
    assert bench.job_throughput(1, 1 << 20, 1.0) == (1 << 20) * 1e3
    assert bench.job_throughput(4, 1 << 20, 2.0) == 2 * (1 << 20) * 1e3


def test_reference_arm_under_torchrun_prints_one_line():
    env = dict(os.environ, PYTHONPATH=ROOT)
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--n-particles", "4096"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["steps"] == 1 and d["warmup"] == 3  # K as given; W raised to the minimum of 3
    assert d["config"]["oracle_sample_particles"] == 4096
