"""The replica (N > 1) path of bench.py on CPU: two gloo ranks, each timing
its own replica; the job's time is the slowest rank's and its throughput sums
all ranks' work.  The reference arm runs on rank 0 only."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 20.0][rank]
    t = bench.max_over_ranks(local_ms, torch, dist, world, torch.device("cpu"))
    rate = bench.job_rate(1000, 10, world, t)
    dist.barrier()
    out.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 20.0
        assert rate == pytest.approx(1000 * 10 * 2 / 0.020)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_oracle_timing_on_several_host_cores():
    """The CPU baseline's all-cores form: one single-threaded oracle process
    per core, each on its own copy of the strip sample, stepped in lock step;
    the rate counts every process's node-updates."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.host_procs() >= 1
    v, n, secs = bench.run_oracle_all_cores(1.0, 1, 0, 2)
    nodes = len(bench.oracle_sample()["mesh"]["xy"])
    assert n == 1 and secs > 0.0
    assert v == pytest.approx(2 * nodes * n / secs)
