"""Long explicit pairs on the packed band pipeline (two pairs per warp, one
per 16-bit half, values relative to a moving per-half base), against the
oracle and against the int32 band pipeline (DSA_LONG_INT32=1).

The packed kernel pairs long pairs by query length; the cases give the two
halves of a unit different query lengths (different band counts, rows past
the shorter pair's end in a shared band), different window lengths (columns
past the shorter window), an odd number of pairs (a unit with an empty
half), lengths that are not multiples of the 512-row bands or the 32-column
blocks, every free-end set, and scores far outside int16 in both
directions (the relative encoding, not the absolute value, has to fit).
Local pairs keep only each band's best and the start state of the 32-step
block that first reached it, and a second kernel reruns that block to find
the first cell holding the pair's maximum; the tie cases put equal maxima in
several bands, several columns and lanes whose columns lag the block.
"""
import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

from test_gpu_parity import assert_same, check_traceback
from test_oracle_bruteforce import MODES

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def packed_fill(monkeypatch):
    """Tracebacks here take the packed fill whatever the band count (the
    library picks it only for calls whose bands fill the device twice)."""
    monkeypatch.setenv("DSA_TB_FILL", "packed")


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


def _run(ctx, qs, db, pairs, S, o, e, mode, fe, trace=True):
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, pairs=pairs)
    if trace:
        ctx.traceback(r)
    ctx.sync()
    return r


def _ragged_set(rng, mode_seed):
    """Seven pairs of 2,100-4,700 residues: related and unrelated targets,
    windows shorter and longer than their queries, one window cut out of
    the middle of a longer target."""
    lens = [4700, 4100, 2100, 3333, 2500, 4096, 2049]
    qs, ts = [], []
    for k, L in enumerate(lens):
        a = rng.integers(0, 4, L).astype(np.uint8)
        if k % 3 == 2:
            t = rng.integers(0, 4, int(L * 0.8) + 17).astype(np.uint8)
        else:
            t = W.mutate(rng, a, 0.04, 0.02)
        qs.append(a)
        ts.append(np.concatenate([rng.integers(0, 4, 300).astype(np.uint8), t,
                                  rng.integers(0, 4, 200).astype(np.uint8)]))
    qset, tset = W.SeqSet.from_list(qs), W.SeqSet.from_list(ts)
    pairs = np.zeros(len(lens), dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.arange(len(lens))
    pairs["target_id"] = np.arange(len(lens))
    pairs["t_offset"] = 300
    pairs["t_len"] = tset.lengths - 500
    return qset, tset, pairs


@pytest.mark.parametrize("mode,fe", MODES)
def test_packed_long_pairs_match_oracle_and_int32(ctx, mode, fe, monkeypatch):
    rng = np.random.default_rng(2000 + 16 * mode + fe)
    qs, db, pairs = _ragged_set(rng, mode)
    S = W.dna_matrix(2, -3)
    assert (qs.lengths * pairs["t_len"].astype(np.int64) >= (1 << 22)).sum() >= 5
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    monkeypatch.delenv("DSA_LONG_INT32", raising=False)
    r16 = _run(ctx, qs, db, pairs, S, 5, 2, mode, fe)
    h16 = r16.hits()
    assert_same((h16["score"], h16["q_end"], h16["t_end"]), (sc, qe, te), f"packed mode={mode} fe={fe}")
    check_traceback(h16, r16.cigar(), qs, db, S, 5, 2, mode, fe)
    monkeypatch.setenv("DSA_LONG_INT32", "1")
    r32 = _run(ctx, qs, db, pairs, S, 5, 2, mode, fe)
    h32 = r32.hits()
    for f in ("score", "q_end", "t_end", "q_begin", "t_begin", "cigar_len"):
        assert np.array_equal(h16[f], h32[f]), f
    assert np.array_equal(r16.cigar(), r32.cigar())


@pytest.mark.parametrize("name,S,o,e", [
    ("dna_1_-4_6_1", W.dna_matrix(1, -4), 6, 1),
    ("o_eq_e", W.dna_matrix(2, -3), 3, 3),
    ("e_zero", W.dna_matrix(2, -3), 4, 0),
    ("smax_zero", np.array([[0, -3, -3, -3], [-3, 0, -3, -3], [-3, -3, 0, -3], [-3, -3, -3, 0]], np.int8), 2, 1),
    ("smax_neg", np.array([[-1, -4, -4, -4], [-4, -1, -4, -4], [-4, -4, -1, -4], [-4, -4, -4, -1]], np.int8), 2, 1),
    ("big_match", W.dna_matrix(9, -2), 10, 1),
    ("asym", np.array([[2, -3, -1, -4], [-2, 3, -3, -1], [-1, -4, 2, -2], [-3, -1, -2, 1]], np.int8), 5, 2),
])
@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15), (dsa.SEMIGLOBAL, 10)])
def test_packed_long_pairs_scoring_corners(ctx, name, S, o, e, mode, fe):
    """Scoring corner cases (every S <= 0, o == e, e == 0, large matches,
    an asymmetric matrix) on three pairs (one unit with an empty half)."""
    rng = np.random.default_rng(2100 + len(name) + 31 * mode + fe)
    a = rng.integers(0, 4, 2300).astype(np.uint8)
    qs = W.SeqSet.from_list([a, rng.integers(0, 4, 2100).astype(np.uint8), a[200:2250]])
    db = W.SeqSet.from_list([W.mutate(rng, a, 0.04, 0.03), rng.integers(0, 4, 2050).astype(np.uint8),
                             W.mutate(rng, a[150:], 0.02, 0.02)])
    pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 2]
    pairs["target_id"] = [0, 1, 2]
    pairs["t_len"] = db.lengths
    r = _run(ctx, qs, db, pairs, S, o, e, mode, fe)
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, o, e, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"{name} mode={mode}")
    check_traceback(h, r.cigar(), qs, db, S, o, e, mode, fe)


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15), (dsa.SEMIGLOBAL, 15)])
def test_packed_long_pairs_scores_far_past_int16(ctx, mode, fe):
    """A near-identical pair of 30,000 residues (+2 a match: scores near
    60,000) next to an unrelated pair of 40,000 against 8,000 residues
    (global score near -56,000): the relative values stay small while the
    absolute ones do not."""
    rng = np.random.default_rng(2200 + mode + fe)
    S = W.dna_matrix(2, -3)
    a = rng.integers(0, 4, 30000).astype(np.uint8)
    b = rng.integers(0, 4, 40000).astype(np.uint8)
    qs = W.SeqSet.from_list([a, b])
    db = W.SeqSet.from_list([W.mutate(rng, a, 0.002, 0.0005), rng.integers(0, 4, 8000).astype(np.uint8)])
    pairs = np.zeros(2, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1]
    pairs["target_id"] = [0, 1]
    pairs["t_len"] = db.lengths
    r = _run(ctx, qs, db, pairs, S, 5, 2, mode, fe, trace=False)
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"far mode={mode}")
    assert sc[0] > 50000
    if mode == dsa.GLOBAL:
        assert sc[1] < -32768


def test_packed_long_pairs_workload_sample(ctx, monkeypatch):
    """Twelve pairs of the long-pair generator (log-uniform 1e4-3e4): scores
    and ends of all against the oracle, both kernels equal including CIGARs."""
    wl = W.long_pairs(seed=W.SEED_BASE + 2300, n_pairs=12, lo=10_000, hi=30_000)
    p = wl.pairs
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes, wl.db.offsets,
                                    p["query_id"], p["target_id"], wl.matrix, 5, 2, wl.mode, 15,
                                    pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    r16 = _run(ctx, wl.queries, wl.db, p, wl.matrix, 5, 2, wl.mode, 15)
    h16 = r16.hits()
    assert_same((h16["score"], h16["q_end"], h16["t_end"]), (sc, qe, te), "workload sample")
    monkeypatch.setenv("DSA_LONG_INT32", "1")
    r32 = _run(ctx, wl.queries, wl.db, p, wl.matrix, 5, 2, wl.mode, 15)
    h32 = r32.hits()
    for f in ("score", "q_end", "t_end", "q_begin", "t_begin", "cigar_len"):
        assert np.array_equal(h16[f], h32[f]), f
    assert np.array_equal(r16.cigar(), r32.cigar())


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15), (dsa.LOCAL, 15),
                                     (dsa.SEMIGLOBAL, 5)])
def test_extreme_long_pair_shapes(ctx, mode, fe, monkeypatch):
    """Long pairs of extreme shape in one call: 450,000 query rows against a
    10-column window (880 bands, no base move after column 10), 10 rows
    against 450,000 columns (one band), and a square pair, paired with each
    other in units of the packed kernel (an odd count: one empty half).
    Scores, ends and tracebacks against the oracle, and both kernels equal."""
    rng = np.random.default_rng(2400 + 16 * mode + fe)
    S = W.dna_matrix(2, -3)
    tall = rng.integers(0, 4, 450_000).astype(np.uint8)
    wide_t = rng.integers(0, 4, 450_000).astype(np.uint8)
    sq = rng.integers(0, 4, 2100).astype(np.uint8)
    qs = W.SeqSet.from_list([tall, wide_t[1000:1010], sq])
    db = W.SeqSet.from_list([tall[5000:5010], wide_t, W.mutate(rng, sq, 0.03, 0.01)])
    pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 2]
    pairs["target_id"] = [0, 1, 2]
    pairs["t_len"] = db.lengths
    assert (qs.lengths * pairs["t_len"].astype(np.int64) >= (1 << 22)).all()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    monkeypatch.delenv("DSA_LONG_INT32", raising=False)
    r16 = _run(ctx, qs, db, pairs, S, 5, 2, mode, fe)
    h16 = r16.hits()
    assert_same((h16["score"], h16["q_end"], h16["t_end"]), (sc, qe, te), f"extreme mode={mode} fe={fe}")
    check_traceback(h16, r16.cigar(), qs, db, S, 5, 2, mode, fe)
    monkeypatch.setenv("DSA_LONG_INT32", "1")
    r32 = _run(ctx, qs, db, pairs, S, 5, 2, mode, fe)
    h32 = r32.hits()
    for f in ("score", "q_end", "t_end", "q_begin", "t_begin", "cigar_len"):
        assert np.array_equal(h16[f], h32[f]), f
    assert np.array_equal(r16.cigar(), r32.cigar())


@pytest.mark.parametrize("case", ["repeats_in_bands", "repeats_in_columns", "low_complexity",
                                  "max_in_first_block", "max_near_window_end"])
def test_packed_local_ties(ctx, case, monkeypatch):
    """Local pairs whose maximum is held by many cells: a 700-residue
    segment repeated down the query (equal maxima in several bands, the
    first row wins), repeated along the target (the first column wins), a
    period-3 sequence against itself shifted (ties everywhere), the maximum
    in the first block, and the maximum at the last columns of the window.
    Scores and ends against the oracle and the int32 kernel, tracebacks
    against the oracle."""
    rng = np.random.default_rng(2500 + len(case))
    S = W.dna_matrix(1, -1)
    o, e = 2, 1
    seg = rng.integers(0, 4, 700).astype(np.uint8)
    if case == "repeats_in_bands":
        q = np.concatenate([seg, rng.integers(0, 4, 77).astype(np.uint8), seg, seg,
                            rng.integers(0, 4, 1300).astype(np.uint8), seg])
        t = np.concatenate([rng.integers(0, 4, 900).astype(np.uint8), seg,
                            rng.integers(0, 4, 1200).astype(np.uint8)])
    elif case == "repeats_in_columns":
        q = np.concatenate([rng.integers(0, 4, 1500).astype(np.uint8), seg,
                            rng.integers(0, 4, 400).astype(np.uint8)])
        t = np.concatenate([seg, rng.integers(0, 4, 33).astype(np.uint8), seg, seg,
                            rng.integers(0, 4, 95).astype(np.uint8), seg])
    elif case == "low_complexity":
        q = np.tile(np.array([0, 1, 2], np.uint8), 1400)
        t = np.tile(np.array([1, 2, 0], np.uint8), 1000)
    elif case == "max_in_first_block":
        q = np.concatenate([seg[:20], rng.integers(0, 4, 3000).astype(np.uint8)])
        t = np.concatenate([seg[:20], rng.integers(0, 4, 2500).astype(np.uint8)])
        S = W.dna_matrix(1, -4)
        o, e = 6, 3
    else:
        q = np.concatenate([rng.integers(0, 4, 2600).astype(np.uint8), seg[:200]])
        t = np.concatenate([rng.integers(0, 4, 2200).astype(np.uint8), seg[:200]])
        S = W.dna_matrix(1, -4)
        o, e = 6, 3
    qs = W.SeqSet.from_list([q, t[:2100], q])
    db = W.SeqSet.from_list([t, q[:2300], t])
    pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 2]
    pairs["target_id"] = [0, 1, 2]
    pairs["t_len"] = db.lengths
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, o, e, dsa.LOCAL, 15,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    monkeypatch.delenv("DSA_LONG_INT32", raising=False)
    r16 = _run(ctx, qs, db, pairs, S, o, e, dsa.LOCAL, 15)
    h16 = r16.hits()
    assert_same((h16["score"], h16["q_end"], h16["t_end"]), (sc, qe, te), case)
    check_traceback(h16, r16.cigar(), qs, db, S, o, e, dsa.LOCAL, 15)
    monkeypatch.setenv("DSA_LONG_INT32", "1")
    r32 = _run(ctx, qs, db, pairs, S, o, e, dsa.LOCAL, 15, trace=False)
    h32 = r32.hits()
    for f in ("score", "q_end", "t_end"):
        assert np.array_equal(h16[f], h32[f]), f


@pytest.mark.parametrize("mode,fe", MODES)
@pytest.mark.parametrize("case", ["ragged", "corners"])
def test_packed_traceback_fill_matches_int32_fill(ctx, mode, fe, case, monkeypatch):
    """The packed traceback fill (two traceback bands per warp, values
    relative to a moving base, decisions from borrow-free differences)
    against the int32 fill (DSA_TB_FILL=int32) and the oracle: bands of
    different window widths share a warp, windows end mid-group, the last
    band of a pair is ragged, and an odd band count leaves a half empty."""
    rng = np.random.default_rng(2600 + 16 * mode + fe + len(case))
    if case == "ragged":
        qs, db, pairs = _ragged_set(rng, mode)
        S, o, e = W.dna_matrix(2, -3), 5, 2
    else:
        a = rng.integers(0, 4, 3100).astype(np.uint8)
        qs = W.SeqSet.from_list([a, rng.integers(0, 4, 2077).astype(np.uint8), a[300:2999]])
        db = W.SeqSet.from_list([W.mutate(rng, a, 0.08, 0.04), rng.integers(0, 4, 2600).astype(np.uint8),
                                 W.mutate(rng, a[100:], 0.02, 0.06)])
        pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
        pairs["query_id"] = [0, 1, 2]
        pairs["target_id"] = [0, 1, 2]
        pairs["t_len"] = db.lengths
        S, o, e = np.array([[2, -3, -1, -4], [-2, 3, -3, -1], [-1, -4, 2, -2], [-3, -1, -2, 1]],
                           np.int8), 4, 4
    monkeypatch.setenv("DSA_TB_FILL", "packed")
    r16 = _run(ctx, qs, db, pairs, S, o, e, mode, fe)
    h16 = r16.hits()
    check_traceback(h16, r16.cigar(), qs, db, S, o, e, mode, fe)
    monkeypatch.setenv("DSA_TB_FILL", "int32")
    r32 = _run(ctx, qs, db, pairs, S, o, e, mode, fe)
    h32 = r32.hits()
    for f in ("score", "q_end", "t_end", "q_begin", "t_begin", "cigar_len"):
        assert np.array_equal(h16[f], h32[f]), f
    assert np.array_equal(r16.cigar(), r32.cigar())
