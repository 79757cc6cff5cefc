"""The multi-process path of the benchmark on CPU: two gloo ranks.

With N replicas each rank renders its own frame (independent problems, no exchange in the
data path); the only collective is the max over ranks of the time per step, from which
the whole-job rate is N steps per that time.  The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.job_rate(times[rank], world)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    times = [2.0, 5.0]
    with mp.get_context("spawn").Manager() as m:    # not forked: the oracle's OpenMP threads may be running
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, times, out), nprocs=world, join=True)
        got = dict(out)
    for rank in range(world):
        ms, value = got[rank]
        assert ms == 5.0 and value == pytest.approx(world * 1000.0 / 5.0)


def test_single_process_rate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(4.0, 1) == (4.0, 250.0)


@pytest.mark.timeout(600)
def test_reference_arm_runs_on_rank_zero_only():
    """torchrun with two gloo ranks: exactly one JSON line, from rank 0, for the whole job."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
