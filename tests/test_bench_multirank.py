"""The N > 1 path of bench.py on the CPU with the gloo backend, world size 2.

The library has no multi-GPU path (replicas only): with N ranks every rank
factors its own matrix and the ranks meet only to time the step (maximum of
the per-rank times) and to count launches (sum).  These tests check those
reductions and that, launched the way a multi-GPU run is launched
(torch.distributed.run, one process per rank), the reference arm prints
exactly one JSON line, from rank 0, and every rank exits 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 + rank  # per-rank step times 1.5 s and 2.5 s
        mx = bench.allreduce_max(dist, t)
        sm = bench.allreduce_sum(dist, 100 + rank)
        bench.barrier(dist)
        out[rank] = (mx, sm)
    finally:
        dist.destroy_process_group()


def test_rank_reductions_gloo_world2():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res == {0: (2.5, 201.0), 1: (2.5, 201.0)}


def test_reference_arm_under_torchrun_world2():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--rows", "20000", "--cols", "64", "--panel", "16"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["unit"] == "TFLOP/s" and d["value"] > 0
    assert d["config"]["panel_b"] == 16 and d["config"]["parallelism"] == "replicas"
    assert d["cpu_baseline"]["kind"] == "oracle"
