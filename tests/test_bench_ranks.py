"""Replica (multi-GPU) host logic of bench.py, on CPU with two gloo ranks.

Environments are independent, so N GPUs run N replicas with no collective
on the data path; the only exchange is the job time, the maximum over ranks
of the timed totals, and the job throughput counts every rank's steps.
"""

import json
import os
import socket
import subprocess
import sys
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
import torch.distributed as dist
sys.path.insert(0, os.getcwd())
import bench
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
local_ms = [120.0, 150.0][rank]
job = bench.slowest_rank_ms(local_ms, dist, device="cpu")
print(json.dumps({"rank": rank, "job_ms": job, "value": bench.job_throughput(100, 4, world, job)}), flush=True)
dist.barrier()
dist.destroy_process_group()
"""


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_job_time_is_the_slowest_rank():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], cwd=ROOT, env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["job_ms"] == 150.0
        assert abs(o["value"] - 100 * 4 * 2 / 0.150) < 1e-9


def test_reference_arm_prints_on_rank0_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = SimpleNamespace(workload="larger_fp64", steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
