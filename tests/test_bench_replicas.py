"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The method has no exchange between independent problems, so N GPUs run N
replicas; the job's throughput is the units of all ranks over the slowest
rank's time.  The aggregation and the reference arm's rank handling run
here without a GPU."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    units = [100.0, 300.0][rank]          # problems solved on this rank
    ms = [20.0, 50.0][rank]               # its timed region
    value, ms_max = bench.job_throughput(ws, units, ms)
    bench.barrier(ws)
    q.put((rank, value, ms_max))
    dist.destroy_process_group()


def test_replica_throughput_is_total_units_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms_max in out:
        assert ms_max == 50.0
        assert abs(value - 400.0 / 0.05) < 1e-6


def test_single_rank_throughput():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.job_throughput(1, 10.0, 100.0)
    assert ms == 100.0 and abs(value - 100.0) < 1e-12


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm prints on rank 0; other ranks exit 0 without work."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "DoF/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
