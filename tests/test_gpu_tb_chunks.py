"""Traceback batches that span several chunks of decision memory.

A traceback call splits its hits into launches whose decision matrices stay
under a word limit (4 GiB for short hits, 32 GiB for long pairs and big
hits).  DSA_TB_CHUNK_WORDS lowers that limit so that small batches cross it.
Each case traces one result with the default limit and the same result
again with the lowered one: the chunked run must launch more kernels, and
its begins, ends and CIGAR words must equal the unchunked run's and the
oracle's (the alignment object's location and CIGAR, Sec. II.B.1).
"""
import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

from test_gpu_parity import check_traceback

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


def _traced(ctx, d, q, S, o, e, mode, fe, monkeypatch, limit, **kw):
    """Align, then trace with the given chunk limit (None: the default)."""
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, **kw)
    ctx.sync()
    if limit is None:
        monkeypatch.delenv("DSA_TB_CHUNK_WORDS", raising=False)
    else:
        monkeypatch.setenv("DSA_TB_CHUNK_WORDS", str(limit))
    n0 = ctx.kernel_launches()
    ctx.traceback(r)
    ctx.sync()
    launches = ctx.kernel_launches() - n0
    monkeypatch.delenv("DSA_TB_CHUNK_WORDS", raising=False)
    h, cig = r.hits(), r.cigar()
    r.free()
    return h, cig, launches


def _alignments(h, cig):
    return [(int(x["q_begin"]), int(x["t_begin"]), int(x["q_end"]), int(x["t_end"]),
             cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])].tolist()) for x in h]


def _compare(ctx, d, q, S, o, e, mode, fe, monkeypatch, limit, queries, db, every=1, **kw):
    h1, c1, n1 = _traced(ctx, d, q, S, o, e, mode, fe, monkeypatch, None, **kw)
    h2, c2, n2 = _traced(ctx, d, q, S, o, e, mode, fe, monkeypatch, limit, **kw)
    assert n2 > n1, f"the lowered limit did not split the batch ({n1} vs {n2} launches)"
    assert _alignments(h1, c1) == _alignments(h2, c2)
    check_traceback(h2[::every], c2, queries, db, S, o, e, mode, fe)
    assert (h2["flags"] & dsa.HIT_HAS_TRACEBACK).any()


@pytest.mark.parametrize("staging", ["device", "host"])
def test_thread_per_hit_chunks(ctx, staging, monkeypatch):
    """6,000 reads in 500 bp windows on the thread-per-hit path: about 4 M
    decision words in chunks of at most 400,000 (the device-staged path hands
    a batch over its limit to the host staging, which splits it)."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1")
    monkeypatch.setenv("DSA_TB_HOST_STAGING", "1" if staging == "host" else "0")
    wl = W.reads_vs_windows(seed=W.SEED_BASE + 310, n_reads=6000, ref_len=200_000)
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    _compare(ctx, d, q, wl.matrix, 6, 1, wl.mode, wl.free_ends, monkeypatch, 400_000,
             wl.queries, wl.db, every=4, pairs=wl.pairs)


def test_warp_per_hit_chunks(ctx, monkeypatch):
    """Top-10 protein hits on the warp-per-hit path, a few hits per chunk."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1000000000")
    wl = W.protein_search(seed=W.SEED_BASE + 311, n_queries=6, n_targets=1500, qlo=64, qhi=600)
    d = ctx.load_set(wl.db, 24)
    q = ctx.load_set(wl.queries, 24)
    _compare(ctx, d, q, wl.matrix, 11, 1, dsa.LOCAL, 15, monkeypatch, 30_000, wl.queries, wl.db,
             top_k=10)


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15), (dsa.SEMIGLOBAL, 10)])
def test_long_pair_chunks(ctx, mode, fe, monkeypatch):
    """Long pairs (band pipeline with checkpoints): one pair per chunk."""
    wl = W.long_pairs(seed=W.SEED_BASE + 312 + mode, n_pairs=5, lo=2500, hi=5000, mode=mode)
    assert (wl.queries.lengths * wl.pairs["t_len"].astype(np.int64) >= (1 << 22)).sum() >= 3
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    _compare(ctx, d, q, wl.matrix, 5, 2, mode, fe, monkeypatch, 100_000, wl.queries, wl.db,
             pairs=wl.pairs)


def test_big_hit_chunks(ctx, monkeypatch):
    """Protein hits of 1,200 x 1,200 residues (checkpointed score pass over the
    hit's rectangle, then the long-pair traceback), one hit per chunk."""
    rng = np.random.default_rng(313)
    bg = W.protein_background()
    qs = [rng.choice(20, 1200, p=bg).astype(np.uint8) for _ in range(3)]
    targets = [W.mutate(rng, x, 0.15, 0.02, alphabet=20) for x in qs for _ in range(2)]
    targets += [rng.choice(20, n, p=bg).astype(np.uint8) for n in rng.integers(50, 800, 100)]
    db = W.SeqSet.from_list(targets)
    queries = W.SeqSet.from_list(qs)
    S = W.blosum62()
    d = ctx.load_set(db, 24)
    q = ctx.load_set(queries, 24)
    _compare(ctx, d, q, S, 11, 1, dsa.LOCAL, 15, monkeypatch, 100_000, queries, db, top_k=2)
