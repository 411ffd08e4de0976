"""Host logic of bench.py on CPU: the N > 1 path runs as two gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    out[rank] = (ms, bench.aggregate_glups(1_000_000, 20, ms, world))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_aggregate():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms, glups = out[r]
        assert ms == 15.0
        assert glups == pytest.approx(2 * 1_000_000 * 20 / 15e-3 / 1e9)


def test_single_rank_aggregate():
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.aggregate_glups(100, 10, 1.0, 1) == pytest.approx(1e-3)


def test_reference_arm_prints_one_json_line():
    """--impl reference times the FP64 oracle on the host and prints one line."""
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "GLUPS"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
