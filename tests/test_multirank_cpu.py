"""The replicas path of bench.py (one process per GPU, no data exchange) on CPU ranks with the
gloo backend, world size 2: the whole-job aggregation (slowest rank's time, all ranks'
units) and the reference arm's rank-0-only output under torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _aggregate_rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.aggregate(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_takes_max_time_and_sum_of_units():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_aggregate_rank, args=(2, free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == (15.0, 300.0)


def test_aggregate_without_process_group_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(3.0, 7.0, None, None) == (3.0, 7.0)


def test_reference_arm_under_torchrun_prints_once():
    """Rank 0 times the oracle and prints the line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "transport2d"]
    env = dict(os.environ, OMP_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")   # CPU ranks (gloo) on any machine
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
