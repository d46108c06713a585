"""The N > 1 path of bench.py on CPU: two gloo ranks.

Each rank builds its shard of one database with the bench's own
`make_workload` (the same queries on every rank, shard r holding global
targets r * targets ...), scores and traces it -- here the oracle stands in
for the rank's GPU -- and hands its top-K hits and CIGAR words to the
bench's `gather_merge`, the partition top-K reduce of Sec. II.B.2.  Rank 0's
merged list must equal the oracle's top K over the whole database (both
shards), hit by hit and CIGAR word by CIGAR word.  The bench's time and
work reductions (slowest rank, summed cells) are checked alongside."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
import numpy as np
import bench
import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

world, rank, local = bench.dist_setup(None, backend="gloo")
assert world == 2 and rank == int(os.environ["RANK"])

args = type("A", (), {"workload": "protein_search", "queries": 3, "targets": 60})()
K = 7

def topk_traced(wl, base):
    # top K per query of the shard by the definition (score desc, id asc),
    # each hit traced by the oracle; ids local to the shard
    S, o, e = wl.matrix, wl.gap_open, wl.gap_extend
    sc, qe, te = oracle.score_all_vs_all(wl.queries, wl.db, S, o, e)
    nq, nt = sc.shape
    hits = np.zeros(nq * K, dtype=dsa.HIT_DTYPE)
    cig = []
    for q in range(nq):
        order = np.lexsort((np.arange(nt), -sc[q]))[:K]
        for r, t in enumerate(order):
            h = hits[q * K + r]
            h["score"], h["q_end"], h["t_end"] = sc[q, t], qe[q, t], te[q, t]
            h["query_id"], h["target_id"] = q, t
            qb, tb, c = oracle.traceback(wl.queries.seq(q), wl.db.seq(int(t)), S, o, e,
                                         oracle.LOCAL, 15, int(qe[q, t]), int(te[q, t]))
            h["q_begin"], h["t_begin"] = qb, tb
            h["flags"] = dsa.HIT_HAS_TRACEBACK
            h["cigar_off"], h["cigar_len"] = len(cig), len(c)
            cig += c.tolist()
    return hits, np.array(cig, np.uint32)

wl = bench.make_workload(args, rank)
assert wl.meta["target_base"] == rank * args.targets and wl.db.n == args.targets
hits, cig = topk_traced(wl, wl.meta["target_base"])
got = bench.gather_merge(world, rank, hits, cig, wl.queries.n, K, wl.meta["target_base"])

ms, cells, gcups = bench.aggregate(world, [1000.0, 1500.0][rank], [3e12, 2e12][rank])
res = {"rank": rank, "ms": ms, "cells": cells, "gcups": gcups,
       "queries": wl.queries.codes.tolist(), "shard": [int(x) for x in wl.db.lengths[:20]]}
if rank == 0:
    assert got is not None
    mh, mc = got
    # the whole database: shard 0 then shard 1 (regenerated here)
    w1 = bench.make_workload(args, 1)
    whole = W.SeqSet.from_list([wl.db.seq(k) for k in range(wl.db.n)] +
                               [w1.db.seq(k) for k in range(w1.db.n)])
    ref = W.Workload("whole", wl.queries, whole, wl.matrix, wl.gap_open, wl.gap_extend, wl.mode)
    want, wc = topk_traced(ref, 0)
    fields = ("score", "q_end", "t_end", "q_begin", "t_begin", "query_id", "target_id")
    res["same_hits"] = all(np.array_equal(mh[f], want[f]) for f in fields)
    res["same_cigars"] = all(
        mc[int(a["cigar_off"]):int(a["cigar_off"]) + int(a["cigar_len"])].tolist() ==
        wc[int(b["cigar_off"]):int(b["cigar_off"]) + int(b["cigar_len"])].tolist()
        for a, b in zip(mh, want))
    res["from_shard_1"] = int((mh["target_id"] >= args.targets).sum())
else:
    assert got is None
print(json.dumps(res))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_shard_search_and_merge_like_the_bench():
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-3000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for o in outs:
        assert o["ms"] == 1500.0
        assert o["cells"] == 5e12
        assert abs(o["gcups"] - 5e12 / 1.5 / 1e9) < 1e-6
    # the same queries on both ranks, different shards of the database
    assert outs[0]["queries"] == outs[1]["queries"]
    assert outs[0]["shard"] != outs[1]["shard"]
    r0 = outs[0]
    assert r0["same_hits"] and r0["same_cigars"]
    assert 0 < r0["from_shard_1"] < 3 * 7
