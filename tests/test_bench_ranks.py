"""The N > 1 path of bench.py on CPU, with world_size 2 and the gloo backend.

The reconstruction does not shard: each rank runs an independent replica of
the scan, the job's time is the slowest rank's (max over ranks) and the
whole-job throughput is the ranks' units over that time.  Under torchrun only
rank 0 prints the JSON line.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 (r + 1) ms: every rank must see the slowest, 20 ms
        m = bench.max_over_ranks(10.0 * (rank + 1), dist)
        with open(os.path.join(out_dir, "rank%d" % rank), "w") as f:
            f.write(repr(m))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_world_size_2(tmp_path):
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    got = [float(open(tmp_path / ("rank%d" % r)).read()) for r in range(2)]
    assert got == [20.0, 20.0]


def test_replica_throughput():
    assert bench.max_over_ranks(3.5) == 3.5
    # two replicas of 100 rows each in 0.02 s (slowest rank)
    assert bench.replica_throughput(2, 100, 0.02) == 10000.0


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--config", "tiny", "--ref-sample", "2000"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["value"] == d["value"]
