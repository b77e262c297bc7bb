"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks stand in for
two GPUs running independent replicas.  The job time is the slowest rank's
(max over ranks after a barrier), the whole-job value counts every rank's
units, and only rank 0 prints the JSON line."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import os, sys, json
import torch
import torch.distributed as dist
sys.path.insert(0, os.environ["ROOT"])
import bench
dist.init_process_group("gloo", rank=int(os.environ["RANK"]), world_size=2)
rank = dist.get_rank()
dist.barrier()
local_ms = 100.0 + 50.0 * rank          # rank 1 is the slow one
t = bench.job_time_ms(dist, local_ms, torch.device("cpu"))
value = bench.job_value(2, 1.0e9, t / 4)
if rank == 0:
    print(json.dumps({"time": t, "value": value}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_max_time_and_whole_job_value():
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    line = json.loads(outs[0][0].strip())
    assert outs[1][0].strip() == ""                    # only rank 0 prints
    assert line["time"] == 150.0                       # the slowest rank
    # 4 steps in 150 ms, 1e9 units per rank per step, 2 ranks: 2e9 / 0.0375 s
    assert abs(line["value"] - 2 * 1.0e9 / 0.0375 / 1e9) < 1e-9


def test_single_process_time_and_value():
    import bench

    assert bench.job_time_ms(None, 12.5, None) == 12.5
    assert bench.job_value(1, 38272753, 71.3) == pytest.approx(38272753 / 0.0713 / 1e9)
