"""Parity at the full benchmark sizes, on outputs the oracle can compute one by one.

* protein search, 32 queries x 500,000 targets: every score and end cell of a
  seeded sample of targets (all queries), the top-10 of every query against
  the dense all-pairs result, and the traceback of every reported hit;
* 1,000,000 reads in 500 bp windows: a seeded sample of 1,500 reads, score,
  ends, begins and CIGAR; every read planted without a mutation scores
  exactly its length with one M run starting at its true origin;
* 64 long DNA pairs (1e4-1e5), global and local: every pair of at most 4e8
  cells in full against the oracle (score, ends, begins, CIGAR), and for
  every pair the CIGAR rescored under the gap rule equals the reported score
  and spans begin..end.
"""
import concurrent.futures as cf

import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


def test_protein_search_full_size(ctx):
    import torch
    wl = W.protein_search()
    d = ctx.load_set(wl.db, 24)
    q = ctx.load_set(wl.queries, 24)
    # dense all-pairs result (packed kernel + wavefront kernel + reruns), kept on the device
    dense = ctx.align(d, q, wl.matrix, 11, 1, flags=dsa.RESULTS_ON_DEVICE)
    ctx.sync()
    dh = dense.device_hits().view(-1, dsa.HIT_DTYPE.itemsize)
    rng = np.random.default_rng(8)
    sample = np.sort(rng.choice(wl.db.n, size=300, replace=False))
    # also the longest targets (they run on the wavefront kernel)
    sample = np.unique(np.concatenate([sample, np.argsort(wl.db.lengths)[-40:]]))
    idx = (torch.arange(wl.queries.n, device="cuda")[:, None] * wl.db.n
           + torch.as_tensor(sample, device="cuda")[None, :]).reshape(-1)
    got = dh.index_select(0, idx).cpu().numpy().view(dsa.HIT_DTYPE).reshape(wl.queries.n, -1)
    sc, qe, te = oracle.score_all_vs_all(wl.queries, wl.db, wl.matrix, 11, 1, targets=sample)
    assert (got["score"] == sc).all() and (got["q_end"] == qe).all() and (got["t_end"] == te).all()
    # top-10 against the dense scores
    scores = dh[:, :4].contiguous().view(torch.int32).reshape(wl.queries.n, wl.db.n).cpu().numpy()
    dense.free()
    r = ctx.align(d, q, wl.matrix, 11, 1, top_k=10)
    ctx.traceback(r)
    ctx.sync()
    h = r.hits().reshape(wl.queries.n, 10)
    for qi in range(wl.queries.n):
        order = np.lexsort((np.arange(wl.db.n), -scores[qi]))[:10]
        assert h["target_id"][qi].tolist() == order.tolist()
    cig = r.cigar()
    for x in r.hits():
        qs_ = wl.queries.seq(int(x["query_id"]))
        ts_ = wl.db.seq(int(x["target_id"]))
        qb, tb, c = oracle.traceback(qs_, ts_, wl.matrix, 11, 1, oracle.LOCAL, 15, int(x["q_end"]),
                                     int(x["t_end"]))
        got_c = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb) and got_c.tolist() == c.tolist()


def test_reads_in_windows_full_size(ctx):
    wl = W.reads_vs_windows()
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 6, 1, mode=dsa.SEMIGLOBAL, free_ends=wl.free_ends, pairs=wl.pairs)
    ctx.traceback(r)
    ctx.sync()
    h = r.hits()
    cig = r.cigar()
    rng = np.random.default_rng(9)
    pick = np.sort(rng.choice(len(wl.pairs), size=1500, replace=False))
    p = wl.pairs[pick]
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes, wl.db.offsets,
                                    p["query_id"], p["target_id"], wl.matrix, 6, 1, oracle.SEMIGLOBAL,
                                    wl.free_ends, pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    hs = h[pick]
    assert (hs["score"] == sc).all() and (hs["q_end"] == qe).all() and (hs["t_end"] == te).all()
    for k in range(0, len(pick), 5):
        x = hs[k]
        qs_ = wl.queries.seq(int(x["query_id"]))
        ts_ = wl.db.codes[int(x["t_offset"]):int(x["t_offset"]) + 500]
        qb, tb, c = oracle.traceback(qs_, ts_, wl.matrix, 6, 1, oracle.SEMIGLOBAL, wl.free_ends,
                                     int(x["q_end"]), int(x["t_end"]))
        got_c = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb) and got_c.tolist() == c.tolist()
    # reads that carry no mutation score exactly their length (match +1) with
    # one M run from their true origin; no read scores more than its length
    lens = wl.queries.lengths
    assert (h["score"] <= lens).all()
    clean = wl.meta["clean"]
    assert clean.sum() > 50_000
    hc = h[clean]
    assert (hc["score"] == lens[clean]).all()
    assert ((hc["t_offset"] + hc["t_begin"].astype(np.uint64)).astype(np.int64)
            == wl.meta["origins"][clean]).all()
    assert (hc["q_begin"] == 0).all() and (hc["cigar_len"] == 1).all()
    assert (cig[hc["cigar_off"].astype(np.int64)] == (lens[clean].astype(np.uint32) << 4)).all()


@pytest.mark.parametrize("mode", [dsa.GLOBAL, dsa.LOCAL])
def test_long_pairs_full_size(ctx, mode):
    wl = W.long_pairs(mode=mode)
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 5, 2, mode=mode, pairs=wl.pairs)
    ctx.traceback(r)
    ctx.sync()
    h = r.hits()
    cig = r.cigar()
    # the oracle's walk (12 bytes per cell of host memory) for every pair of at
    # most 4e8 cells, three pairs at a time
    sizes = wl.queries.lengths * wl.pairs["t_len"].astype(np.int64)
    small = [int(k) for k in np.argsort(sizes) if sizes[k] <= 400_000_000]
    assert len(small) >= 10
    p = wl.pairs[small]
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix, 5, 2,
                                    mode, 15)
    assert (h["score"][small] == sc).all() and (h["q_end"][small] == qe).all()
    assert (h["t_end"][small] == te).all()

    def walk(k):
        return oracle.traceback(wl.queries.seq(k), wl.db.seq(k), wl.matrix, 5, 2, mode, 15,
                                int(h["q_end"][k]), int(h["t_end"][k]))

    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        for k, (qb, tb, c) in zip(small, ex.map(walk, small)):
            got_c = cig[int(h["cigar_off"][k]):int(h["cigar_off"][k]) + int(h["cigar_len"][k])]
            assert (int(h["q_begin"][k]), int(h["t_begin"][k])) == (qb, tb), k
            assert got_c.tolist() == c.tolist(), k
    for k, x in enumerate(h):
        c = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        ln = (c >> 4).astype(np.int64)
        op = c & 15
        nq = int(ln[op != 2].sum()); nt = int(ln[op != 1].sum())
        assert (int(x["q_begin"]) + nq - 1, int(x["t_begin"]) + nt - 1) == (int(x["q_end"]), int(x["t_end"]))
        qs_ = wl.queries.seq(k)[int(x["q_begin"]):]
        ts_ = wl.db.seq(k)[int(x["t_begin"]):]
        m_ops = op == 0
        # rescore: matches/mismatches along M runs, gap runs o + (k-1)e
        total = 0
        i = j = 0
        for L, o_ in zip(ln, op):
            if o_ == 0:
                total += int((np.where(qs_[i:i + L] == ts_[j:j + L], 2, -3)).sum())
                i += L; j += L
            elif o_ == 1:
                total -= 5 + (L - 1) * 2; i += L
            else:
                total -= 5 + (L - 1) * 2; j += L
        assert total == int(x["score"]), k
        if mode == dsa.GLOBAL:
            assert (int(x["q_begin"]), int(x["t_begin"])) == (0, 0)
