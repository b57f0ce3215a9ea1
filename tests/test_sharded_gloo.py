"""Row-sharded generations of one population over two ranks (CPU, gloo).

One population does not split into independent parts: every row draws its
donors from the whole population (Eq. 1, Alg. 2), so a rank that owns rows
[r N / P, (r + 1) N / P) needs every row of the previous generation. The
protocol checked here is the one a multi-GPU build would run, with the
oracle standing in for each rank's generation kernel:

  1. every rank holds the whole population and fitness of generation g;
  2. rank r makes generation g for its own rows only (donors from all rows,
     the draws of (seed, g, i) as everywhere, so ownership changes no draw);
  3. the ranks exchange only what changed: the indices, rows and fitness of
     their accepted trials (an all-gather of variable-length lists);
  4. every rank writes the gathered rows into its copy: generation g + 1.

The populations and fitness values of every rank after each generation
must equal, bit for bit, those of the unsharded oracle, for uneven shard
sizes (N not a multiple of the rank count) and each crossover.
"""
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
import numpy as np
import torch.distributed as dist
import oracle as O
from paper_2101_06599_gb300 import workloads as W

dist.init_process_group("gloo")
r, P = dist.get_rank(), dist.get_world_size()
out = {"rank": r, "ok": True, "sent": 0, "checked": 0}
for xo in ("nec", "bin", "exp"):
    N, D, F, CR, seed, obj = 37, 23, 0.5, 0.9, 7, "rastrigin"
    lo, hi = W.BOXES[obj]
    pop = W.population(N, D, lo, hi, 3)
    fit = O.evaluate(obj, pop)
    ref_pop, ref_fit = pop.copy(), fit.copy()
    i0, i1 = (r * N) // P, ((r + 1) * N) // P            # uneven shards
    for g in range(6):
        s = O.step(pop, fit, F, CR, xo, obj, lo, hi, seed, g, rows=(i0, i1), want_trial=False)
        mine = [(i, s.pop[i].tobytes().hex(), float(s.fit[i])) for i in range(i0, i1) if s.accept[i - i0]]
        out["sent"] += len(mine)
        gathered = [None] * P
        dist.all_gather_object(gathered, mine)
        for lst in gathered:
            for i, row, f in lst:
                pop[i] = np.frombuffer(bytes.fromhex(row), dtype=np.float32)
                fit[i] = f
        u = O.step(ref_pop, ref_fit, F, CR, xo, obj, lo, hi, seed, g, want_trial=False)
        ref_pop, ref_fit = u.pop, u.fit
        same = (np.array_equal(pop.view(np.uint32), ref_pop.view(np.uint32))
                and np.array_equal(fit.view(np.uint64), ref_fit.view(np.uint64)))
        out["ok"] = out["ok"] and bool(same)
        out["checked"] += 1
print(json.dumps(out), flush=True)
dist.destroy_process_group()
"""


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_row_sharded_generations_match_the_unsharded_oracle(world):
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER, ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e[-2000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for d in outs:
        assert d["ok"], d
        assert d["checked"] == 18
    assert sum(d["sent"] for d in outs) > 0
