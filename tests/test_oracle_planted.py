"""Pin the oracle to reads planted in a genome (read-vs-window workload).

A read copied from the genome without any mutation, aligned semi-globally
(target ends free) inside a window that contains its source slice, scores
exactly its length times the match score: every read residue can earn at
most one match and any gap costs, so the optimum is the gapless exact copy.
Its traceback is one M run that starts at the read's true origin.  These
facts come from the construction of the reads, not from any DP.
"""
import numpy as np

import oracle
from paper_1701_01575_gb300 import workloads as W


def test_clean_reads_score_their_length_at_their_origin():
    wl = W.reads_vs_windows(seed=W.SEED_BASE + 500, n_reads=600, ref_len=60_000)
    clean = wl.meta["clean"]
    origins = wl.meta["origins"]
    assert 30 < clean.sum() < len(clean)
    p = wl.pairs
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix, 6, 1,
                                    oracle.SEMIGLOBAL, wl.free_ends, pair_toff=p["t_offset"],
                                    pair_tlen=p["t_len"])
    lens = wl.queries.lengths
    assert (sc[clean] == lens[clean]).all()
    # a mutated read never beats its length
    assert (sc <= lens).all()
    for k in np.flatnonzero(clean)[:40]:
        w0 = int(p["t_offset"][k])
        window = wl.db.codes[w0:w0 + int(p["t_len"][k])]
        qb, tb, cig = oracle.traceback(wl.queries.seq(k), window, wl.matrix, 6, 1,
                                       oracle.SEMIGLOBAL, wl.free_ends, int(qe[k]), int(te[k]))
        assert (qb, w0 + tb) == (0, int(origins[k]))
        assert cig.tolist() == [int(lens[k]) << 4 | oracle.OP_M]
