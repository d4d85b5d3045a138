"""The N > 1 host path of bench.py on CPU: world-size-2 gloo ranks.

Every rank of a multi-GPU run is an independent replica (the products shard
into independent problems, with no data-path exchange); what crosses ranks is
the barrier, the maximum of the timed durations and rank 0's single line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 40.25][rank]
    got = bench.max_over_ranks(ms, dist)
    dist.barrier()
    out[rank] = (got, bench.job_rate(world, 1e12, 5, got))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        got, rate = res[r]
        assert got == 40.25
        # whole-job rate: 2 ranks x 5 steps x 1e12 units over the slowest rank
        assert rate == pytest.approx(2 * 5 * 1e12 / 0.04025)


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, None) == 3.5


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line():
    """--impl reference at N = 2: rank 0 times the oracle and prints one line;
    rank 1 exits 0 without work."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
