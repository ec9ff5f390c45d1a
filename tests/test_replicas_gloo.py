"""The N > 1 path on CPU: world-size-2 gloo ranks.

Runs on several GPUs are independent replicas: the ranks share only the
clock (a barrier on both sides, the slowest rank's time) and add up their
units.  These tests run that logic as two gloo processes, and the reference
arm of the benchmark under torchrun, where rank 0 alone works and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2305_13380_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.barrier()
        # rank r processes 100 (r + 1) units in (r + 1) ms
        rate, ms = replicas.job_throughput(100.0 * (rank + 1), 1.0 + rank)
        out.put((rank, replicas.world_size(), rate, ms, replicas.max_over_ranks(-rank)))
        replicas.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, rate, ms, mx in got:
        assert world == 2
        assert ms == 2.0                       # the slowest rank's time
        assert rate == pytest.approx(300.0 / 2e-3)  # all units over that time
        assert mx == 0.0


def test_replicas_without_a_process_group():
    from paper_2305_13380_gb300 import replicas
    assert not replicas.active()
    assert replicas.world_size() == 1
    replicas.barrier()
    assert replicas.job_throughput(50.0, 10.0) == (5000.0, 10.0)


def test_reference_arm_under_torchrun_prints_once():
    # two ranks: rank 0 times the oracle and prints one line, rank 1 exits 0
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "lattice8", "--ref-budget", "1"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
