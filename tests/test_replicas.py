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


def test_line_summary_is_short_and_tolerates_skipped_parts():
    """The bench line ends with a compact summary of its ratios (a reader keeping only the
    line's end still has them); with the forms and configurations skipped it still forms."""
    sys.path.insert(0, ROOT)
    import bench
    stages = {"project": 0.0355, "bin_sort": 0.1667, "render_fwd": 0.322, "loss": 0.0593, "render_bwd": 0.5049,
              "project_bwd": 0.0512, "pose+dsr+step": 0.0284}
    roof = {k: {"bound": "hbm", "frac": 0.3} for k in stages}
    roof["time_weighted_frac"] = 0.25
    forms = {"single_fp32": {"frames_per_s": 916.9}, "batched_fp32": {"frames_per_s": 1127.1},
             "batched_f16rgb_bf16feat": {"frames_per_s": 1117.5}}
    configs = {"batching_24_keyframes": {"ms_per_step": 16.15},
               "precision_2M_d32_bf16_f16": {"ms_per_step": 12.80, "speedup_vs_fp32": 1.027},
               "precision_2M_d32_fp32": {"ms_per_step": 13.14},
               "differentiation_1M_d32_640x480": {"ms_per_step": 0.763}}
    s = bench.summary(stages, roof, forms, configs, {"ms_per_frame": 25.3})
    assert s["half_vs_batched_fp32"] == round(1117.5 / 1127.1, 3)
    assert s["precision_2M_d32_half_vs_fp32"] == 1.027
    assert s["forms_frames_per_s"]["batched_fp32"] == 1127.1
    assert "time_weighted_frac" not in s["stages_frac"]
    assert len(json.dumps(s)) < 1000
    bare = bench.summary(stages, roof, None, None, None)
    assert set(bare) == {"stages_ms", "stages_frac"}
