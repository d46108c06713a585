"""Partition + reduce of top-K lists (Sec. II.B.2): the merge of exact
per-partition lists equals the top K of the whole database under the order
score descending, target id ascending.  Host logic: no GPU needed."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1701_01575_gb300 import build, dsa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    dsa.load_library()


def topk_lists(score, qend, tend, k, base=0, cig_tag=None):
    """Top-k per query of a score matrix by the definition: sort by (score
    descending, target id ascending); ids local to the matrix.  With cig_tag,
    every hit gets one CIGAR word naming its (tag, global target)."""
    nq, nt = score.shape
    kk = min(k, nt)
    hits = np.zeros(nq * kk, dtype=dsa.HIT_DTYPE)
    cig = []
    for q in range(nq):
        order = np.lexsort((np.arange(nt), -score[q]))[:kk]
        for r, t in enumerate(order):
            h = hits[q * kk + r]
            h["score"], h["q_end"], h["t_end"] = score[q, t], qend[q, t], tend[q, t]
            h["query_id"], h["target_id"] = q, t
            if cig_tag is not None:
                h["flags"] = 2   # DSA_HIT_HAS_TRACEBACK
                h["cigar_off"], h["cigar_len"] = len(cig), 2
                cig += [((base + t) << 4) | 0, (cig_tag << 4) | 1]
    return hits, (np.array(cig, np.uint32) if cig_tag is not None else None)


@pytest.mark.parametrize("seed,k,cuts", [(0, 10, [0, 7, 8, 40, 100]), (1, 5, [0, 3, 6, 9, 60]),
                                         (2, 64, [0, 100]), (3, 10, [0, 50, 100])])
def test_merge_equals_global_topk(seed, k, cuts):
    rng = np.random.default_rng(seed)
    nq, nt = 6, cuts[-1]
    score = rng.integers(0, 6, (nq, nt)).astype(np.int32)   # many ties
    qend = rng.integers(0, 100, (nq, nt)).astype(np.int32)
    tend = rng.integers(0, 100, (nq, nt)).astype(np.int32)
    parts = []
    for p in range(len(cuts) - 1):
        a, b = cuts[p], cuts[p + 1]
        parts.append(topk_lists(score[:, a:b], qend[:, a:b], tend[:, a:b], k, base=a, cig_tag=p))
    got, cig = dsa.merge_topk(parts, cuts[:-1], nq, k)
    want, _ = topk_lists(score, qend, tend, k)
    for f in ("score", "q_end", "t_end", "query_id", "target_id"):
        assert np.array_equal(got[f], want[f]), f
    # every CIGAR followed its hit: its first word names the global target
    for h in got:
        w = cig[h["cigar_off"]:h["cigar_off"] + h["cigar_len"]]
        assert len(w) == 2 and (int(w[0]) >> 4) == int(h["target_id"])
        part = np.searchsorted(cuts, int(h["target_id"]), side="right") - 1
        assert (int(w[1]) >> 4) == part


def test_merge_rejects_bad_lists():
    rng = np.random.default_rng(9)
    s = rng.integers(0, 50, (2, 20)).astype(np.int32)
    z = np.zeros_like(s)
    good, _ = topk_lists(s, z, z, 4)
    bad = good.copy()
    bad[[0, 1]] = bad[[1, 0]]                       # out of rank order
    if bad["score"][0] != bad["score"][1] or bad["target_id"][0] != bad["target_id"][1]:
        with pytest.raises(dsa.DsaError, match="top-K order"):
            dsa.merge_topk([(bad, None)], [0], 2, 4)
    wrong_q = good.copy()
    wrong_q["query_id"][5] = 0
    with pytest.raises(dsa.DsaError, match="belongs to query"):
        dsa.merge_topk([(wrong_q, None)], [0], 2, 4)
    with pytest.raises(dsa.DsaError, match="multiple"):
        dsa.merge_topk([(good[:7], None)], [0], 2, 4)
    traced, cig = topk_lists(s, z, z, 4, cig_tag=0)
    with pytest.raises(dsa.DsaError, match="CIGAR"):
        dsa.merge_topk([(traced, None)], [0], 2, 4)


CHILD = r"""
import os, sys, json
sys.path.insert(0, os.environ["ROOT"])
sys.path.insert(0, os.path.join(os.environ["ROOT"], "tests"))
import numpy as np
import torch.distributed as dist
from paper_1701_01575_gb300 import dsa, workloads as W
from oracle import oracle
from test_merge_topk import topk_lists
dist.init_process_group("gloo", init_method="env://")
rank, world = dist.get_rank(), dist.get_world_size()
rng = np.random.default_rng(77)
bg = W.protein_background()
db = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8) for n in rng.integers(20, 120, 61)])
qs = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8) for n in rng.integers(10, 60, 4)])
S, k = W.blosum62(), 8
# this rank's shard: a contiguous range of targets, scored by the oracle
cuts = [0, 25, db.n]
a, b = cuts[rank], cuts[rank + 1]
shard = db.subset(np.arange(a, b))
sc, qe, te = oracle.score_all_vs_all(qs, shard, S, 11, 1)
hits, _ = topk_lists(sc, qe, te, k)
lists = [None] * world
dist.all_gather_object(lists, hits.tobytes())
ok = True
if rank == 0:
    parts = [(np.frombuffer(x, dtype=dsa.HIT_DTYPE), None) for x in lists]
    got, _ = dsa.merge_topk(parts, cuts[:-1], qs.n, k)
    sc, qe, te = oracle.score_all_vs_all(qs, db, S, 11, 1)
    want, _ = topk_lists(sc, qe, te, k)
    ok = all(np.array_equal(got[f], want[f]) for f in ("score", "q_end", "t_end", "target_id"))
print(json.dumps({"rank": rank, "ok": bool(ok)}))
dist.destroy_process_group()
"""


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_sharded_search_reduce_two_gloo_ranks():
    """Each gloo rank scores its shard of the database (the oracle stands in
    for a device), the ranks exchange their top-K lists, and rank 0's merge
    equals the oracle's top K over the whole database."""
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, ROOT=ROOT, RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    for p in procs:
        out, err = p.communicate(timeout=240)
        assert p.returncode == 0, err[-3000:]
        assert json.loads(out.strip().splitlines()[-1])["ok"]
