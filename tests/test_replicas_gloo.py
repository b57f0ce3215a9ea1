"""The multi-process side of bench.py (one replica per rank, `replicas
only`) on CPU with the gloo backend, world size 2: the max and sum over
ranks that form the whole-job value, distinct replica seeds, and a
non-zero rank of the reference arm leaving at once without output."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
import torch
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
bench._dist = dist
r = dist.get_rank()
bench.barrier()
out = {"rank": r, "world": dist.get_world_size(),
       "max": bench.max_over_ranks(torch, 10.0 * (r + 1)),
       "sum": bench.sum_over_ranks(torch, 1.5 + r),
       "seed": bench.replica_seed(r)}
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_reduce_and_seed():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    for d in outs:
        assert d["world"] == 2
        assert d["max"] == 20.0 and d["sum"] == 4.0
    assert outs[0]["seed"] != outs[1]["seed"]


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "3", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""
