"""The multi-GPU path is replicas: each rank runs its own copy of the
workload and the job's rate is all ranks' points over the slowest rank's
time.  Checked here with two gloo ranks on the CPU: the barrier and the
max-over-ranks reduction of bench.py, the reported rate, and the reference
arm printing from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    barrier, max_over_ranks = bench.make_collectives(dist, world, torch.device("cpu"))
    barrier()
    ms_local = 100.0 + 50.0 * rank               # the second rank is slower
    ms = max_over_ranks(ms_local)
    rate = bench.replica_rate(world, 1000, 5, ms)
    out[rank] = (ms, rate)
    barrier()
    dist.destroy_process_group()


def test_replicas_max_over_ranks_and_rate():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 150.0                        # every rank sees the slowest time
        assert abs(rate - world * 1000 * 5 / 0.150) < 1e-6


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1", "--points", "2000", "--face-points", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "1", "--points", "2000", "--face-points", "0"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
