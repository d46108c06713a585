"""The N > 1 control path of bench.py on CPU: two gloo ranks.

Each rank reports its own time and cells; the job's time is the slowest
rank's, its work the sum, and its throughput their ratio (weak scaling: each
rank aligns its own database shard).  No data-path collective exists."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import bench
world, rank, local = bench.dist_setup(None, backend="gloo")
assert world == 2 and rank == int(os.environ["RANK"])
bench.barrier(world)
ms_local = [1000.0, 1500.0][rank]
cells_local = [3e12, 2e12][rank]
ms, cells, gcups = bench.aggregate(world, ms_local, cells_local)
wl = bench.make_workload(type("A", (), {"workload": "protein_search", "queries": 2, "targets": 50})(), rank)
print(json.dumps({"rank": rank, "ms": ms, "cells": cells, "gcups": gcups,
                  "shard": [int(x) for x in wl.db.lengths[:20]]}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_aggregate_like_the_bench():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-3000:]
        outs.append(__import__("json").loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 1500.0
        assert o["cells"] == 5e12
        assert abs(o["gcups"] - 5e12 / 1.5 / 1e9) < 1e-6
    # each rank draws its own database shard
    assert outs[0]["shard"] != outs[1]["shard"]
