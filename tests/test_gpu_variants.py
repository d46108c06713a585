"""Kernel variants of the packed kernels and their autotuner.

The inter-sequence kernels exist for two strip heights (28 rows, and 20 rows
that waste fewer padding rows on short queries); the explicit-pairs kernel's
byte form for two (16 rows at 4 blocks per SM, 20 rows at 3); the long-pair
band pipeline runs at 2 or 4 blocks per SM.  Every variant
must give the oracle's scores and end cells bit for bit in every mode; the
tuner times the variants on the first call of a workload shape and records
its choice (and the long-target threshold) in its cache file, which the
next call reads.
"""
import json

import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

from test_gpu_parity import assert_same, gpu_all, oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("rows", ["28", "20"])
@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 10), (dsa.SEMIGLOBAL, 5)])
def test_strip_height_variants_match_oracle(ctx, rows, mode, fe, monkeypatch):
    """Query lengths around both strip heights and many queries per lane
    stream; every target on the inter-sequence kernel."""
    monkeypatch.setenv("DSA_INTER_ROWS", rows)
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "1000000")
    rng = np.random.default_rng(1200 + int(rows) + 16 * mode + fe)
    bg = W.protein_background()
    qlens = [1, 19, 20, 21, 27, 28, 29, 39, 40, 41, 56, 57, 60, 61, 140] + \
        [int(x) for x in rng.integers(1, 90, 20)]
    queries = W._make_set(rng, qlens, bg)
    db = W._make_set(rng, rng.integers(1, 260, 300), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"rows={rows} mode={mode} fe={fe}")
    assert g[5].phase_cells()["inter16"] > 0


@pytest.mark.parametrize("rows", ["28", "20"])
def test_strip_height_variants_saturation(ctx, rows, monkeypatch):
    """The saturation flag and int32 rerun in both variants (local)."""
    monkeypatch.setenv("DSA_INTER_ROWS", rows)
    w = W.PROTEIN_LETTERS.index("W")
    run = np.full(3100, w, np.uint8)
    rng = np.random.default_rng(1250)
    bg = W.protein_background()
    queries = W.SeqSet.from_list([run, rng.choice(20, 77, p=bg).astype(np.uint8)])
    db = W.SeqSet.from_list([run, rng.choice(20, 300, p=bg).astype(np.uint8)])
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1)
    g = gpu_all(ctx, queries, db, S, 11, 1)
    assert_same(g[:3], orc, f"rows={rows}")
    assert g[0][0, 0] == 3100 * 11 and g[4] >= 1


@pytest.mark.parametrize("mode", [dsa.LOCAL, dsa.GLOBAL])
def test_tuner_records_variant_and_reuses_it(ctx, mode, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSA_AUTOTUNE_CACHE", str(cache))
    monkeypatch.setenv("DSA_AUTOTUNE", "retune")
    monkeypatch.delenv("DSA_INTER_ROWS", raising=False)
    monkeypatch.delenv("DSA_LONG_THRESHOLD", raising=False)
    rng = np.random.default_rng(1300 + mode)
    bg = W.protein_background()
    queries = W._make_set(rng, rng.integers(20, 60, 12), bg)
    db = W._make_set(rng, rng.integers(30, 400, 3000), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode)
    assert_same(g[:3], orc, "tuned")
    entries = json.loads(cache.read_text())
    rows = {k: v for k, v in entries.items() if k.endswith("|rows")}
    assert len(rows) == 1 and list(rows.values())[0] in (20, 28)
    key = list(rows)[0]
    assert ("|local|" in key) == (mode == dsa.LOCAL)
    assert key[:-len("|rows")] + "|thr" in entries
    # a cached choice is reused: the next call does not tune (same result,
    # cache unchanged)
    monkeypatch.setenv("DSA_AUTOTUNE", "cache")
    before = cache.read_text()
    g2 = gpu_all(ctx, queries, db, S, 11, 1, mode=mode)
    assert_same(g2[:3], orc, "cached")
    assert cache.read_text() == before


@pytest.mark.parametrize("rows", ["16", "20"])
@pytest.mark.parametrize("mode,fe", [(dsa.SEMIGLOBAL, 12), (dsa.LOCAL, 15), (dsa.GLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 15)])
def test_pairs_kernel_variants_match_oracle(ctx, rows, mode, fe, monkeypatch):
    """The packed pairs kernel's byte form in both strip heights (16 rows at
    4 blocks per SM, 20 rows at 3): reads of 1-300 bp in windows, strips
    ragged against both heights."""
    monkeypatch.setenv("DSA_PAIRS_ROWS", rows)
    rng = np.random.default_rng(1400 + int(rows) + 16 * mode + fe)
    genome = rng.integers(0, 4, 60_000).astype(np.uint8)
    lens = np.concatenate([[1, 15, 16, 17, 19, 20, 21, 39, 40, 41], rng.integers(1, 300, 600)])
    reads, starts = [], []
    for n in lens:
        st = int(rng.integers(0, 60_000 - 700))
        r = W.mutate(rng, genome[st + 50: st + 50 + int(n)], 0.03, 0.02)
        reads.append(r if len(r) else np.zeros(1, np.uint8))
        starts.append(st)
    qs = W.SeqSet.from_list(reads)
    db = W.SeqSet.from_list([genome])
    pairs = np.zeros(qs.n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.arange(qs.n)
    pairs["t_offset"] = starts
    pairs["t_len"] = 400 + rng.integers(0, 200, qs.n)
    S = W.dna_matrix(1, -4)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 6, 1, mode=mode, free_ends=fe, pairs=pairs)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 6, 1, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"rows={rows}")
    assert r.phase_cells()["inter16"] > 0


def test_pairs_tuner_records_variant(ctx, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSA_AUTOTUNE_CACHE", str(cache))
    monkeypatch.setenv("DSA_AUTOTUNE", "retune")
    monkeypatch.delenv("DSA_PAIRS_ROWS", raising=False)
    wl = W.reads_vs_windows(seed=W.SEED_BASE + 1450, n_reads=4000, ref_len=100_000)
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 6, 1, mode=wl.mode, free_ends=wl.free_ends, pairs=wl.pairs)
    ctx.sync()
    h = r.hits()
    p = wl.pairs
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix, 6, 1,
                                    wl.mode, wl.free_ends, pair_toff=p["t_offset"],
                                    pair_tlen=p["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "tuned pairs")
    entries = json.loads(cache.read_text())
    keys = [k for k in entries if "|pairs|" in k]
    assert len(keys) == 1 and entries[keys[0]] in (16, 20)


@pytest.mark.parametrize("blocks", ["2", "4"])
@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15), (dsa.SEMIGLOBAL, 10)])
def test_long_pair_blocks_per_sm_variants(ctx, blocks, mode, fe, monkeypatch):
    """The long-pair band pipeline with 2 or 4 blocks per SM (a persistent
    grid smaller than the band items: warps take several bands in turn)."""
    monkeypatch.setenv("DSA_LONG_BLOCKS", blocks)
    wl = W.long_pairs(seed=W.SEED_BASE + 1500 + mode + fe, n_pairs=9, lo=3000, hi=9000, mode=mode)
    p = wl.pairs
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 5, 2, mode=mode, free_ends=fe, pairs=p)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix, 5, 2,
                                    mode, fe, pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"blocks={blocks} mode={mode}")
    assert r.phase_cells()["intra16"] > 0


def test_long_pair_tuner_records_blocks(ctx, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSA_AUTOTUNE_CACHE", str(cache))
    monkeypatch.setenv("DSA_AUTOTUNE", "retune")
    monkeypatch.delenv("DSA_LONG_BLOCKS", raising=False)
    wl = W.long_pairs(seed=W.SEED_BASE + 1550, n_pairs=6, lo=3000, hi=9000)
    p = wl.pairs
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 5, 2, mode=wl.mode, pairs=p)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], wl.matrix, 5, 2,
                                    wl.mode, 15, pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "tuned long pairs")
    entries = json.loads(cache.read_text())
    keys = [k for k in entries if "|long|" in k]
    assert len(keys) == 1 and entries[keys[0]] in (2, 4)
