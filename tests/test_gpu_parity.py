"""GPU parity: libdsa (through the C ABI) against the CPU oracle, element by element.

Scores, end cells, begin cells and CIGARs are integers: the bar is bit-exact.
Sizes span several strips (32 query rows), interleave chunks (16 residues),
warp groups (32 targets) and CTA blocks (8 groups), with ragged tails.
"""
import zlib

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


def oracle_all(queries, db, S, o, e, mode=oracle.LOCAL, fe=15):
    return oracle.score_all_vs_all(queries, db, S, o, e, mode, fe)


def gpu_all(ctx, queries, db, S, o, e, mode=dsa.LOCAL, fe=15, flags=0, A=None):
    A = A or S.shape[0]
    d = ctx.load_set(db, A)
    q = ctx.load_set(queries, A)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, flags=flags)
    ctx.sync()
    h = r.hits()
    cells, rerun = r.stats()
    shape = (queries.n, db.n)
    assert (h["query_id"].reshape(shape) == np.arange(queries.n)[:, None]).all()
    assert (h["target_id"].reshape(shape) == np.arange(db.n)[None, :]).all()
    return (h["score"].reshape(shape), h["q_end"].reshape(shape), h["t_end"].reshape(shape),
            h["flags"].reshape(shape), rerun, r)


def assert_same(gpu, orc, what=""):
    for name, g, o_ in zip(("score", "q_end", "t_end"), gpu, orc):
        bad = np.argwhere(g != o_)
        assert len(bad) == 0, f"{what} {name}: {len(bad)} mismatches, first {bad[:5].tolist()} " \
                              f"gpu={g[tuple(bad[0])]} oracle={o_[tuple(bad[0])]}"


# ---------------------------------------------------------------- local, packed path

def test_protein_vs_db_full(ctx):
    """1 query (128) vs 2,000 targets U{50..500}, BLOSUM62 11/1, local."""
    wl = W.protein_vs_db()
    orc = oracle_all(wl.queries, wl.db, wl.matrix, 11, 1)
    for flags in (0, dsa.FORCE_INT32, dsa.PLAIN_FORM):
        g = gpu_all(ctx, wl.queries, wl.db, wl.matrix, 11, 1, flags=flags)
        assert_same(g[:3], orc, f"flags={flags}")


def test_protein_search_small(ctx):
    """Odd query count, lengths across strip boundaries, many groups, ragged tails."""
    rng = np.random.default_rng(11)
    bg = W.protein_background()
    qlens = np.array([1, 27, 28, 29, 31, 32, 33, 56, 57, 64, 65, 200, 517, 95])
    queries = W._make_set(rng, qlens, bg)
    tl = np.concatenate([rng.integers(1, 40, 300), rng.integers(40, 700, 2500),
                         [1, 15, 16, 17, 2000, 1999]])
    db = W._make_set(rng, tl, bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1)
    g = gpu_all(ctx, queries, db, S, 11, 1)
    assert_same(g[:3], orc, "packed")
    assert g[4] == 0


@pytest.mark.parametrize("seed", [1, 2])
def test_query_streams_many_queries(ctx, seed):
    """Many queries of mixed lengths: each 16-bit half runs a stream of several queries."""
    rng = np.random.default_rng(70 + seed)
    S = W.dna_matrix(2, -3)
    lens = np.concatenate([rng.integers(1, 40, 12), rng.integers(30, 140, 8), [32, 64, 96, 33, 1]])
    queries = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8) for n in lens])
    db = W.random_dna(rng, 520, 1, 260)
    orc = oracle_all(queries, db, S, 4, 1)
    g = gpu_all(ctx, queries, db, S, 4, 1)
    assert_same(g[:3], orc, "streams")


@pytest.mark.parametrize("thr", ["0", "64", "100000"])
def test_long_target_threshold_variants(ctx, thr, monkeypatch):
    """Targets above the threshold run on the wavefront kernel; every split is bit-exact."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", thr)
    rng = np.random.default_rng(12)
    bg = W.protein_background()
    queries = W._make_set(rng, np.array([1, 16, 31, 33, 300, 511, 512, 513, 700]), bg)
    db = W._make_set(rng, np.concatenate([rng.integers(1, 200, 150), [1, 63, 64, 65, 1500, 900]]), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1)
    g = gpu_all(ctx, queries, db, S, 11, 1)
    assert_same(g[:3], orc, f"thr={thr}")
    cells = g[5].phase_cells()
    if thr == "0":
        assert cells["inter16"] == 0 and cells["intra16"] == g[5].stats()[0]
    if thr == "100000":
        assert cells["intra16"] == 0


@pytest.mark.parametrize("o,e", [(1, 0), (5, 2), (3, 3)])
def test_long_targets_wavefront_ties(ctx, o, e, monkeypatch):
    """Multi-band queries (> 512 rows) against long DNA targets; small alphabet forces ties."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "256")
    rng = np.random.default_rng(200 + o + e)
    S = W.dna_matrix(2, -3)
    queries = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8) for n in (1, 40, 513, 1100, 1030)])
    tl = [rng.integers(0, 4, n).astype(np.uint8) for n in rng.integers(257, 2500, 40)]
    tl += [W.mutate(rng, queries.seq(3), 0.05, 0.02)]
    db = W.SeqSet.from_list(tl)
    orc = oracle_all(queries, db, S, o, e)
    g = gpu_all(ctx, queries, db, S, o, e)
    assert_same(g[:3], orc, f"o={o} e={e}")
    assert g[5].phase_cells()["intra16"] > 0


@pytest.mark.parametrize("o,e", [(1, 0), (3, 3), (5, 2), (12, 1), (40, 7)])
def test_local_gap_params_and_ties(ctx, o, e):
    """Small alphabets force many ties: exercises the (j, i) end-cell rule."""
    rng = np.random.default_rng(100 + o * 10 + e)
    S = W.dna_matrix(2, -3)
    queries = W.random_dna(rng, 5, 1, 120)
    db = W.random_dna(rng, 700, 1, 300)
    orc = oracle_all(queries, db, S, o, e)
    g = gpu_all(ctx, queries, db, S, o, e)
    assert_same(g[:3], orc, f"o={o} e={e}")


def test_asymmetric_matrix_orientation(ctx):
    """Rows of S are query residues, columns target residues."""
    rng = np.random.default_rng(5)
    S = rng.integers(-6, 7, size=(7, 7)).astype(np.int8)
    queries = W._make_set(rng, rng.integers(1, 90, 4), np.full(7, 1 / 7))
    db = W._make_set(rng, rng.integers(1, 200, 400), np.full(7, 1 / 7))
    orc = oracle_all(queries, db, S, 4, 1)
    for flags in (0, dsa.FORCE_INT32):
        g = gpu_all(ctx, queries, db, S, 4, 1, flags=flags)
        assert_same(g[:3], orc, f"flags={flags}")


def test_all_zero_local(ctx):
    S = np.full((4, 4), -1, dtype=np.int8)
    q = W.SeqSet.from_list([np.zeros(40, np.uint8)])
    db = W.SeqSet.from_list([np.ones(n, np.uint8) for n in (1, 5, 70)])
    g = gpu_all(ctx, q, db, S, 3, 1)
    assert (g[0] == 0).all() and (g[1] == -1).all() and (g[2] == -1).all()


def test_saturation_rerun_exact_long(ctx, monkeypatch):
    """Saturation flagged by the wavefront kernel too."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "0")
    test_saturation_rerun_exact(ctx)


def test_saturation_rerun_exact(ctx):
    """Scores above the int16 range: flagged by the packed pass, rerun exactly in int32."""
    w = W.PROTEIN_LETTERS.index("W")
    rng = np.random.default_rng(3)
    bg = W.protein_background()
    run = np.full(3500, w, np.uint8)
    queries = W.SeqSet.from_list([run, rng.choice(20, 300, p=bg).astype(np.uint8), run[:100]])
    db = W.SeqSet.from_list([run, np.concatenate([rng.choice(20, 50, p=bg).astype(np.uint8), run]),
                             rng.choice(20, 400, p=bg).astype(np.uint8), run[:2990]])
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1)
    g = gpu_all(ctx, queries, db, S, 11, 1)
    assert_same(g[:3], orc, "saturation")
    assert g[0][0, 0] == 3500 * 11 and g[0][0, 1] == 3500 * 11
    assert g[4] >= 3 and (g[3][0, :2] & dsa.HIT_RERUN_INT32).all()


# ---------------------------------------------------------------- other modes (int32 path)

@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15), (dsa.SEMIGLOBAL, 12),
                                     (dsa.SEMIGLOBAL, 3), (dsa.SEMIGLOBAL, 9), (dsa.SEMIGLOBAL, 0)])
def test_global_semiglobal_all_vs_all(ctx, mode, fe):
    rng = np.random.default_rng(7 + fe)
    bg = W.protein_background()
    queries = W._make_set(rng, rng.integers(1, 70, 3), bg)
    db = W._make_set(rng, rng.integers(1, 150, 300), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 10, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 10, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe}")


def test_explicit_pairs_reads_in_windows(ctx):
    wl = W.reads_vs_windows(n_reads=3000, ref_len=200_000)
    S = wl.matrix
    p = wl.pairs
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes,
                                    wl.db.offsets, p["query_id"], p["target_id"], S, 6, 1,
                                    oracle.SEMIGLOBAL, wl.free_ends, pair_toff=p["t_offset"],
                                    pair_tlen=p["t_len"])
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, S, 6, 1, mode=dsa.SEMIGLOBAL, free_ends=wl.free_ends, pairs=p)
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "pairs")
    assert (h["t_offset"] == p["t_offset"]).all()


# ---------------------------------------------------------------- top-k and traceback

def test_topk_order(ctx):
    rng = np.random.default_rng(21)
    S = W.dna_matrix(1, -1)   # many tied scores
    queries = W.random_dna(rng, 3, 10, 40)
    db = W.random_dna(rng, 1500, 5, 60)
    sc, qe, te = oracle_all(queries, db, S, 2, 1)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(queries, 4)
    for k in (1, 10, 16, 40):
        r = ctx.align(d, q, S, 2, 1, top_k=k)
        h = r.hits().reshape(queries.n, k)
        for qi in range(queries.n):
            order = sorted(range(db.n), key=lambda t: (-sc[qi, t], t))[:k]
            assert h["target_id"][qi].tolist() == order
            assert h["score"][qi].tolist() == [sc[qi, t] for t in order]
            assert h["q_end"][qi].tolist() == [qe[qi, t] for t in order]


def check_traceback(h, cig, queries, db, S, o, e, mode, fe):
    for x in h:
        q = queries.seq(int(x["query_id"]))
        t = db.seq(int(x["target_id"]))[int(x["t_offset"]):]
        if mode == oracle.LOCAL and x["score"] == 0:
            assert x["cigar_len"] == 0
            continue
        qb, tb, c = oracle.traceback(q, t, S, o, e, mode, fe, int(x["q_end"]), int(x["t_end"]))
        got = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb)
        assert got.tolist() == c.tolist(), (oracle.cigar_string(got), oracle.cigar_string(c))


@pytest.mark.parametrize("per_thread", [False, True])
@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 12), (dsa.SEMIGLOBAL, 3)])
def test_traceback_matches_oracle(ctx, mode, fe, per_thread, monkeypatch):
    """Warp-per-hit and thread-per-hit traceback (the latter forced on small batches)."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1" if per_thread else "1000000000")
    rng = np.random.default_rng(31 + mode + fe)
    S = W.dna_matrix(2, -3)
    base = W.random_dna(rng, 4, 20, 400)
    # related targets: mutated copies, so alignments have gaps
    tl = []
    for k in range(60):
        src = base.seq(k % base.n)
        tl.append(W.mutate(rng, src, 0.08, 0.04) if k % 3 else rng.integers(0, 4, 50).astype(np.uint8))
    tl = [x if len(x) else np.zeros(1, np.uint8) for x in tl]
    db = W.SeqSet.from_list(tl)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(base, 4)
    r = ctx.align(d, q, S, 5, 2, mode=mode, free_ends=fe)
    ctx.traceback(r)
    h = r.hits()
    check_traceback(h, r.cigar(), base, db, S, 5, 2, mode, fe)
    assert (h["flags"] & dsa.HIT_HAS_TRACEBACK).sum() >= len(h) // 2


def test_traceback_topk_protein_long_hits(ctx):
    """Hits spanning several traceback bands (256 rows) and wide targets."""
    rng = np.random.default_rng(41)
    bg = W.protein_background()
    q0 = rng.choice(20, 900, p=bg).astype(np.uint8)
    targets = [W.mutate(rng, q0, 0.2, 0.02, alphabet=20) for _ in range(6)]
    targets += [rng.choice(20, n, p=bg).astype(np.uint8) for n in rng.integers(50, 1200, 200)]
    db = W.SeqSet.from_list(targets)
    queries = W.SeqSet.from_list([q0, rng.choice(20, 300, p=bg).astype(np.uint8)])
    S = W.blosum62()
    d = ctx.load_set(db, 24)
    q = ctx.load_set(queries, 24)
    r = ctx.align(d, q, S, 11, 1, top_k=10)
    ctx.traceback(r)
    h = r.hits()
    check_traceback(h, r.cigar(), queries, db, S, 11, 1, oracle.LOCAL, 15)
    assert h["score"][0] > 1000


def test_issue_probe(ctx):
    for form in range(12):
        rate = ctx.probe_issue_rate(form)
        assert 0.05 < rate < 16, (form, rate)
    with pytest.raises(dsa.DsaError) as ex:
        ctx.probe_issue_rate(12)
    assert ex.value.code == dsa.ERR_INVALID_ARG


def test_memory_budget_enforced():
    c = dsa.Context(0, mem_budget=1 << 20)
    rng = np.random.default_rng(0)
    db = W.random_dna(rng, 10, 200_000, 200_000)
    with pytest.raises(dsa.DsaError) as ei:
        c.load_set(db, 4)
    assert ei.value.code == dsa.ERR_OVER_BUDGET
    c.close()


def test_bad_arguments_rejected(ctx):
    rng = np.random.default_rng(0)
    db = W.random_dna(rng, 10, 5, 50)
    with pytest.raises(dsa.DsaError):
        ctx.load(np.array([0, 1, 9], np.uint8), np.array([0, 3], np.uint64), 4)   # code >= A
    d = ctx.load_set(db, 4)
    with pytest.raises(dsa.DsaError):
        ctx.align(d, d, W.dna_matrix(1, -1), 1, 2)                               # e > o
    with pytest.raises(dsa.DsaError):
        ctx.align(d, d, W.blosum62(), 1, 1)                                      # A mismatch


# ---------------------------------------------------------------- long explicit pairs

@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15), (dsa.SEMIGLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 12), (dsa.SEMIGLOBAL, 3), (dsa.SEMIGLOBAL, 10)])
def test_long_pairs_banded_score_and_traceback(ctx, mode, fe):
    """Pairs of 2,000-6,000 bp (band pipeline across warps, checkpointed traceback)."""
    wl = W.long_pairs(seed=W.SEED_BASE + 30 + mode, n_pairs=5, lo=2000, hi=6000, mode=mode)
    p = wl.pairs
    assert (wl.queries.lengths * p["t_len"].astype(np.int64) >= (1 << 22)).any()
    sc, qe, te = oracle.score_pairs(wl.queries.codes, wl.queries.offsets, wl.db.codes, wl.db.offsets,
                                    p["query_id"], p["target_id"], wl.matrix, 5, 2, mode, fe,
                                    pair_toff=p["t_offset"], pair_tlen=p["t_len"])
    d = ctx.load_set(wl.db, 4)
    q = ctx.load_set(wl.queries, 4)
    r = ctx.align(d, q, wl.matrix, 5, 2, mode=mode, free_ends=fe, pairs=p)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"long mode={mode}")
    assert r.phase_cells()["intra16"] > 0
    ctx.traceback(r)
    ctx.sync()
    check_traceback(r.hits(), r.cigar(), wl.queries, wl.db, wl.matrix, 5, 2, mode, fe)


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 10), (dsa.LOCAL, 15),
                                     (dsa.SEMIGLOBAL, 15), (dsa.SEMIGLOBAL, 3)])
def test_long_pair_traceback_diagonal_band(ctx, mode, fe):
    """Diagonal bands of the long-pair traceback (two-sided for paths from
    (0, 0), one-sided from the end cell otherwise): related pairs (narrow
    band), an unrelated pair (band wider than the target: whole rows), lengths
    not multiples of the 256-row bands, m != n."""
    rng = np.random.default_rng(123 + fe)
    S = W.dna_matrix(2, -3)
    a = rng.integers(0, 4, 3001).astype(np.uint8)
    b = rng.integers(0, 4, 2300).astype(np.uint8)
    qs = W.SeqSet.from_list([a, b, a[:2900]])
    db = W.SeqSet.from_list([W.mutate(rng, a, 0.05, 0.01), rng.integers(0, 4, 2100).astype(np.uint8),
                             W.mutate(rng, a[150:], 0.02, 0.02)])
    pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 2]
    pairs["target_id"] = [0, 1, 2]
    pairs["t_len"] = db.lengths
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 5, 2, mode=mode, free_ends=fe, pairs=pairs)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"long band mode={mode}")
    assert r.phase_cells()["intra16"] == int((qs.lengths * db.lengths).sum())
    ctx.traceback(r)
    ctx.sync()
    check_traceback(r.hits(), r.cigar(), qs, db, S, 5, 2, mode, fe)


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 12), (dsa.LOCAL, 15)])
def test_long_pair_traceback_exact_match_edge(ctx, mode, fe):
    """Error-free long pairs: the score leaves no slack, so the diagonal band
    is the path's own diagonal and the path runs along the edge of every
    band's column window, through the corner cell each band takes from the
    row above it (the boundary row for the first band, a checkpoint row
    after that)."""
    rng = np.random.default_rng(77 + fe)
    S = W.dna_matrix(1, -4)
    g = rng.integers(0, 4, 6000).astype(np.uint8)
    qs = W.SeqSet.from_list([g[100:2200], g[1000:3700], g[3000:5100]])
    db = W.SeqSet.from_list([g[90:2200], g[1000:3700], g[2990:5110]])
    pairs = np.zeros(3, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 2]
    pairs["target_id"] = [0, 1, 2]
    pairs["t_len"] = db.lengths
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 6, 1, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 6, 1, mode=mode, free_ends=fe, pairs=pairs)
    ctx.traceback(r)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"exact long mode={mode}")
    check_traceback(h, r.cigar(), qs, db, S, 6, 1, mode, fe)


def test_long_and_short_pairs_mixed(ctx):
    """One call with pairs on both sides of the banded-path threshold."""
    rng = np.random.default_rng(99)
    S = W.dna_matrix(2, -3)
    a = rng.integers(0, 4, 3000).astype(np.uint8)
    seqs = [a, W.mutate(rng, a, 0.05, 0.01), rng.integers(0, 4, 200).astype(np.uint8)]
    qs = W.SeqSet.from_list([seqs[0], seqs[2]])
    db = W.SeqSet.from_list([seqs[1], seqs[2]])
    pairs = np.zeros(4, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1, 0, 1]
    pairs["target_id"] = [0, 1, 1, 0]
    pairs["t_len"] = [db.lengths[0], db.lengths[1], db.lengths[1], 1500]
    pairs["t_offset"] = [0, 0, 0, 700]
    for mode in (dsa.GLOBAL, dsa.LOCAL):
        sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                        pairs["target_id"], S, 5, 2, mode, 15,
                                        pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
        d = ctx.load_set(db, 4)
        q = ctx.load_set(qs, 4)
        r = ctx.align(d, q, S, 5, 2, mode=mode, pairs=pairs)
        ctx.traceback(r)
        ctx.sync()
        h = r.hits()
        assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"mixed mode={mode}")
        check_traceback(h, r.cigar(), qs, db, S, 5, 2, mode, 15)


# ---------------------------------------------------------------- failure path

@pytest.mark.parametrize("kind", [0, 1])
def test_bounded_wait_gives_up_and_context_survives(ctx, kind):
    """A wait nothing satisfies ends after its limit with DSA_ERR_DEVICE_TIMEOUT; no fault."""
    import time
    t0 = time.time()
    st = ctx.selftest_wait_timeout(kind, 200_000_000)   # 0.2 s
    assert st == dsa.ERR_DEVICE_TIMEOUT
    assert time.time() - t0 < 5
    ctx.sync()   # status cleared
    # the context still aligns correctly
    wl = W.protein_vs_db(n_targets=100)
    g = gpu_all(ctx, wl.queries, wl.db, wl.matrix, 11, 1)
    orc = oracle_all(wl.queries, wl.db, wl.matrix, 11, 1)
    assert_same(g[:3], orc, "after timeout")


# ---------------------------------------------------------------- packed explicit pairs

def _pairs_case(rng, qs, db, n, vary_len=True):
    pairs = np.zeros(n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = rng.integers(0, qs.n, n)
    pairs["target_id"] = rng.integers(0, db.n, n)
    tl = db.lengths[pairs["target_id"].astype(np.int64)]
    off = (rng.random(n) * (tl // 3)).astype(np.int64) if vary_len else np.zeros(n, np.int64)
    pairs["t_offset"] = off
    ln = tl - off
    if vary_len:
        ln = np.maximum(1, ln - (rng.random(n) * ln // 3).astype(np.int64))
    pairs["t_len"] = ln
    return pairs


@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 12), (dsa.SEMIGLOBAL, 3), (dsa.SEMIGLOBAL, 9)])
def test_packed_pairs_all_modes(ctx, mode, fe):
    """Two pairs of equal query length per thread; odd counts, uneven windows, ties."""
    rng = np.random.default_rng(500 + mode * 16 + fe)
    S = W.dna_matrix(2, -3)
    qs = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8)
                             for n in np.concatenate([rng.integers(1, 60, 30), [15, 16, 17, 31, 32, 33]])])
    db = W.random_dna(rng, 40, 20, 300)
    pairs = _pairs_case(rng, qs, db, 901)
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, mode, fe, pair_toff=pairs["t_offset"],
                                    pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 5, 2, mode=mode, free_ends=fe, pairs=pairs)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"packed pairs mode={mode} fe={fe}")
    assert r.phase_cells()["inter16"] > 0
    if mode != dsa.LOCAL:
        ctx.traceback(r)
        check_traceback(r.hits()[:200], r.cigar(), qs, db, S, 5, 2, mode, fe)


def test_packed_pairs_device_plan_multi_digit(ctx):
    """Device planning of a pair list with query and window lengths above 255
    (two sort digits each) over several sort tiles: pairs given from host
    memory and from device memory give the oracle's results."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2024)
    S = W.dna_matrix(2, -3)
    n_q, n_pairs = 900, 6000
    qlen = np.where(rng.random(n_q) < 0.8, rng.integers(1, 81, n_q), rng.integers(250, 651, n_q))
    qs = W.SeqSet.from_list([rng.integers(0, 4, int(n)).astype(np.uint8) for n in qlen])
    db = W.random_dna(rng, 50, 1200, 1400)
    pairs = np.zeros(n_pairs, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = rng.integers(0, n_q, n_pairs)
    pairs["target_id"] = rng.integers(0, db.n, n_pairs)
    tl = np.where(rng.random(n_pairs) < 0.8, rng.integers(1, 121, n_pairs), rng.integers(260, 1101, n_pairs))
    room = db.lengths[pairs["target_id"]] - tl
    pairs["t_offset"] = (rng.random(n_pairs) * (room + 1)).astype(np.uint64)
    pairs["t_len"] = tl
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 5, 2, dsa.SEMIGLOBAL, 12,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    dev = torch.as_tensor(pairs.view(np.uint8), device="cuda")
    for p_arg in (pairs, dev):
        r = ctx.align(d, q, S, 5, 2, mode=dsa.SEMIGLOBAL, free_ends=12, pairs=p_arg)
        ctx.sync()
        h = r.hits()
        assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "device-planned pairs")
        assert (h["query_id"] == pairs["query_id"]).all() and (h["t_offset"] == pairs["t_offset"]).all()
        assert r.phase_cells()["inter16"] == int((qs.lengths[pairs["query_id"]] * tl).sum())
        r.free()


def test_fasta_fastq_ingest_to_alignment(ctx, tmp_path):
    """A FASTA database and FASTQ reads go through the streaming reader, the
    device load and a semi-global search of each read in its window; the
    oracle scores the codes the generator wrote."""
    rng = np.random.default_rng(31)
    genome = [rng.integers(0, 4, int(n)).astype(np.uint8) for n in (5000, 3000)]
    fa = tmp_path / "g.fa"
    with open(fa, "w") as f:
        for k, g in enumerate(genome):
            f.write(f">chr{k}\n")
            text = "".join("ACGT"[c] for c in g)
            for x in range(0, len(text), 61):
                f.write(text[x:x + 61] + "\n")
    reads, pairs = [], np.zeros(40, dtype=W.PAIR_DTYPE)
    for k in range(40):
        t = k % 2
        st = int(rng.integers(0, len(genome[t]) - 300))
        reads.append(W.mutate(rng, genome[t][st + 20: st + 20 + int(rng.integers(50, 150))], 0.02, 0.01))
        pairs[k] = (k, t, st, 250, 0)
    fq = tmp_path / "r.fq"
    with open(fq, "w") as f:
        for k, rd in enumerate(reads):
            f.write(f"@read{k}\n{''.join('ACGT'[c] for c in rd)}\n+\n{'I' * len(rd)}\n")
    with dsa.Reader(path=str(fa), alphabet=dsa.ALPHABET_DNA4, chunk_bytes=1000) as r:
        dcodes, doffs, dnames, _ = r.next_batch()
    qcodes, qoffs, qnames, _ = dsa.read_sequences(path=str(fq), alphabet=dsa.ALPHABET_DNA4)
    db = W.SeqSet.from_list(genome)
    qs = W.SeqSet.from_list(reads)
    assert np.array_equal(dcodes, db.codes) and np.array_equal(qcodes, qs.codes)
    assert dnames == ["chr0", "chr1"] and qnames[7] == "read7"
    d = ctx.load(dcodes, doffs, 4)
    q = ctx.load(qcodes, qoffs, 4)
    S = W.dna_matrix(1, -4)
    r = ctx.align(d, q, S, 6, 1, mode=dsa.SEMIGLOBAL, free_ends=12, pairs=pairs)
    ctx.traceback(r)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 6, 1, dsa.SEMIGLOBAL, 12,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "ingested reads")
    check_traceback(h, r.cigar(), qs, db, S, 6, 1, dsa.SEMIGLOBAL, 12)


@pytest.mark.parametrize("part_res", [0, 9_000, 700, 1])
def test_partitioned_search_equals_whole_database(ctx, part_res):
    """Sec. II.B.2's partition + reduce on one device: the database is loaded
    and searched a partition at a time (top 10, traceback) and the lists are
    merged; hits, coordinates and CIGARs equal one search of the whole
    database (partitions of one target each at the smallest size)."""
    rng = np.random.default_rng(404)
    bg = W.protein_background()
    db = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8)
                             for n in rng.integers(30, 400, 120)])
    qs = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8) for n in (60, 150, 333)])
    S = W.blosum62()
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    whole = ctx.align(d, q, S, 11, 1, top_k=10)
    ctx.traceback(whole)
    want, wcig = whole.hits(), whole.cigar()
    part = ctx.search_partitioned(db.codes, db.offsets, 24, q, S, 11, 1, top_k=10,
                                  partition_residues=part_res)
    got, gcig = part.hits(), part.cigar()
    for f in ("score", "q_begin", "q_end", "t_begin", "t_end", "query_id", "target_id"):
        assert np.array_equal(got[f], want[f]), f
    for a, b in zip(got, want):
        assert np.array_equal(gcig[a["cigar_off"]:a["cigar_off"] + a["cigar_len"]],
                              wcig[b["cigar_off"]:b["cigar_off"] + b["cigar_len"]])
    assert part.stats()[0] == whole.stats()[0]
    with pytest.raises(dsa.DsaError):
        ctx.traceback(part)   # host-only result


def _pssm_case(rng, n_q=5, n_t=150, lo=-8, hi=10):
    bg = W.protein_background()
    qs = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8)
                             for n in rng.integers(20, 260, n_q)])
    db = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8)
                             for n in rng.integers(10, 700, n_t)])
    P = rng.integers(lo, hi + 1, size=(int(qs.offsets[-1]), 24)).astype(np.int8)
    return qs, db, P


@pytest.mark.parametrize("thr", ["4096", "300"])
def test_pssm_search_local_matches_oracle(ctx, thr, monkeypatch):
    """Position-specific scores (Sec. II.C.2 user-defined scoring) on the packed
    local kernels: with a long-target threshold of 300 part of the database
    takes the wavefront kernel; every score and end of the dense matrix equals
    the oracle's."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", thr)
    rng = np.random.default_rng(600 + int(thr))
    qs, db, P = _pssm_case(rng)
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    r = ctx.align_pssm(d, q, P, 11, 1)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_all_vs_all(qs, db, W.blosum62(), 11, 1, pssm=P)
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc.ravel(), qe.ravel(), te.ravel()), "pssm local")
    if thr == "300":
        assert r.phase_cells()["intra16"] > 0
    with pytest.raises(dsa.DsaError) as ex:
        ctx.traceback(r)
    assert ex.value.code == dsa.ERR_UNSUPPORTED


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 12), (dsa.SEMIGLOBAL, 3)])
def test_pssm_search_global_modes_match_oracle(ctx, mode, fe):
    rng = np.random.default_rng(610 + mode + fe)
    qs, db, P = _pssm_case(rng, n_q=3, n_t=60)
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    r = ctx.align_pssm(d, q, P, 11, 1, mode=mode, free_ends=fe)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_all_vs_all(qs, db, W.blosum62(), 11, 1, mode=mode, free_ends=fe, pssm=P)
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc.ravel(), qe.ravel(), te.ravel()), "pssm global")


def test_pssm_saturation_rerun_and_top_k(ctx):
    """A profile that rewards one target's residues with +100 drives the
    packed pass past int16: those pairs are rerun in int32 from the same
    profile.  Top-K follows (score desc, target id asc)."""
    rng = np.random.default_rng(620)
    bg = W.protein_background()
    qs = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8) for n in (400, 90, 150, 33)])
    db = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8)
                             for n in [500 if k == 7 else int(rng.integers(10, 600)) for k in range(80)]])
    P = rng.integers(-3, 4, size=(int(qs.offsets[-1]), 24)).astype(np.int8)
    target = db.seq(7)
    P[np.arange(400), target[:400]] = 100   # query 0 position i likes target 7's residue i
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    r = ctx.align_pssm(d, q, P, 11, 1)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_all_vs_all(qs, db, W.blosum62(), 11, 1, pssm=P)
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc.ravel(), qe.ravel(), te.ravel()), "pssm rerun")
    assert sc[0, 7] > 32767 and r.stats()[1] >= 1
    k = 6
    rk = ctx.align_pssm(d, q, P, 11, 1, top_k=k)
    hk = rk.hits()
    for qi in range(qs.n):
        order = np.lexsort((np.arange(db.n), -sc[qi]))[:k]
        got = hk[qi * k:(qi + 1) * k]
        assert got["target_id"].tolist() == order.tolist()
        assert got["score"].tolist() == sc[qi, order].tolist()


@pytest.mark.parametrize("flags", ["force_int32", "plain_form"])
def test_pssm_search_int32_forms(ctx, flags):
    """Position-specific local search through the exact int32 kernel (every
    pair) and through the plain per-query form: the int32 profile builder
    reads the profile's rows."""
    rng = np.random.default_rng(640 + len(flags))
    qs, db, P = _pssm_case(rng, n_q=3, n_t=70)
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    f = dsa.FORCE_INT32 if flags == "force_int32" else dsa.PLAIN_FORM
    r = ctx.align_pssm(d, q, P, 11, 1, flags=f)
    ctx.sync()
    h = r.hits()
    sc, qe, te = oracle.score_all_vs_all(qs, db, W.blosum62(), 11, 1, pssm=P)
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc.ravel(), qe.ravel(), te.ravel()), flags)
    assert r.phase_cells()["int32"] > 0


def test_pssm_of_the_matrix_equals_matrix_search(ctx):
    """The profile whose row i is S[q_i] gives the matrix search's results
    bit for bit (scores, ends, rerun flags), locally and globally."""
    rng = np.random.default_rng(630)
    qs, db, _ = _pssm_case(rng, n_q=6, n_t=120)
    S = W.blosum62()
    P = S[qs.codes]
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    for mode in (dsa.LOCAL, dsa.GLOBAL):
        a = ctx.align(d, q, S, 11, 1, mode=mode).hits()
        b = ctx.align_pssm(d, q, P, 11, 1, mode=mode).hits()
        for f in ("score", "q_end", "t_end", "flags", "target_id", "query_id"):
            assert np.array_equal(a[f], b[f]), (mode, f)
    with pytest.raises(ValueError):
        ctx.align_pssm(d, q, P[:-1], 11, 1)


def test_partitioned_search_scores_only(ctx):
    """Partition + reduce without traceback: the merged top K (scores, ends,
    global target ids) equals the resident search's and carries no CIGAR."""
    rng = np.random.default_rng(405)
    bg = W.protein_background()
    db = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8)
                             for n in rng.integers(30, 300, 90)])
    qs = W.SeqSet.from_list([rng.choice(20, int(n), p=bg).astype(np.uint8) for n in (40, 120)])
    S = W.blosum62()
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    want = ctx.align(d, q, S, 11, 1, top_k=7).hits()
    part = ctx.search_partitioned(db.codes, db.offsets, 24, q, S, 11, 1, top_k=7,
                                  partition_residues=2_000, traceback=False)
    got = part.hits()
    for f in ("score", "q_end", "t_end", "query_id", "target_id"):
        assert np.array_equal(got[f], want[f]), f
    assert (got["cigar_len"] == 0).all() and len(part.cigar()) == 0


def test_pair_range_errors(ctx):
    """Out-of-range pairs are refused with the smallest bad index, whether the
    pairs are in host or device memory; nothing is aligned."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    qs = W.SeqSet.from_list([rng.integers(0, 4, 30).astype(np.uint8) for _ in range(5)])
    db = W.random_dna(rng, 4, 100, 100)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    S = W.dna_matrix(1, -4)
    good = np.zeros(5000, dtype=W.PAIR_DTYPE)
    good["query_id"] = rng.integers(0, 5, 5000)
    good["target_id"] = rng.integers(0, 4, 5000)
    good["t_len"] = 50
    bad_cases = [("query_id", 5), ("target_id", 4), ("t_len", 0), ("t_len", 101),
                 ("t_offset", 2 ** 63), ("t_offset", 51)]
    for field, value in bad_cases:
        p = good.copy()
        p[field][4321] = value
        p[field][4999] = value
        for p_arg in (p, torch.as_tensor(p.view(np.uint8), device="cuda")):
            with pytest.raises(dsa.DsaError) as ex:
                ctx.align(d, q, S, 6, 1, mode=dsa.SEMIGLOBAL, free_ends=12, pairs=p_arg)
            assert ex.value.code == dsa.ERR_INVALID_ARG
            assert "pair 4321 is out of range" in str(ex.value), (field, value)


def test_packed_pairs_protein_local(ctx):
    rng = np.random.default_rng(42)
    bg = W.protein_background()
    qs = W.SeqSet.from_list([rng.choice(20, n, p=bg).astype(np.uint8) for n in rng.integers(1, 300, 20)])
    db = W.SeqSet.from_list([rng.choice(20, n, p=bg).astype(np.uint8) for n in rng.integers(10, 600, 30)])
    pairs = _pairs_case(rng, qs, db, 500)
    S = W.blosum62()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 11, 1, oracle.LOCAL, 15,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 24)
    q = ctx.load_set(qs, 24)
    r = ctx.align(d, q, S, 11, 1, pairs=pairs)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "protein pairs")
    assert r.phase_cells()["inter16"] > 0


def test_packed_pairs_saturation_rerun(ctx):
    """Local pairs whose best passes 32767 - max S are flagged and rerun in int32."""
    rng = np.random.default_rng(43)
    S = W.dna_matrix(100, -90)
    run = np.zeros(400, np.uint8)
    qs = W.SeqSet.from_list([run, run[:380], rng.integers(0, 4, 380).astype(np.uint8)]
                            + [rng.integers(0, 4, n).astype(np.uint8) for n in rng.integers(1, 200, 10)])
    db = W.SeqSet.from_list([np.concatenate([rng.integers(0, 4, 50).astype(np.uint8), run, run[:7]]),
                             rng.integers(0, 4, 900).astype(np.uint8)])
    pairs = np.zeros(40, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.concatenate([[0, 1, 2], rng.integers(0, qs.n, 37)])
    pairs["target_id"] = np.concatenate([[0, 0, 1], rng.integers(0, 2, 37)])
    pairs["t_offset"] = 0
    pairs["t_len"] = db.lengths[pairs["target_id"].astype(np.int64)]
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 50, 5, oracle.LOCAL, 15,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 50, 5, pairs=pairs)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), "saturating pairs")
    assert h["score"][0] == 40000 and (h["flags"][0] & dsa.HIT_RERUN_INT32)
    assert not (h["flags"][2] & dsa.HIT_RERUN_INT32)
    assert r.stats()[1] >= 2


@pytest.mark.parametrize("staging", ["device", "host"])
@pytest.mark.parametrize("uniform", [False, True])
@pytest.mark.parametrize("mode,fe", [(dsa.SEMIGLOBAL, 12), (dsa.GLOBAL, 15), (dsa.LOCAL, 15),
                                     (dsa.SEMIGLOBAL, 15)])
def test_thread_traceback_reads_in_windows(ctx, mode, fe, uniform, staging, monkeypatch):
    """Thread-per-hit traceback on read/window pairs: 1..70-row reads (one strip,
    several strips, ragged last strip, fewer than 9 rows), partial last group;
    uniform = equal read and window lengths; jobs staged on the device or on
    the host."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1")
    monkeypatch.setenv("DSA_TB_HOST_STAGING", "1" if staging == "host" else "0")
    rng = np.random.default_rng(70 + mode * 16 + fe + 7 * uniform)
    genome = rng.integers(0, 4, 20000).astype(np.uint8)
    db = W.SeqSet.from_list([genome])
    reads, starts = [], []
    lens = np.full(203, 40) if uniform else np.concatenate([rng.integers(1, 71, 200), [1, 8, 9, 16, 17, 32, 33]])
    for n in lens:
        st = int(rng.integers(0, 20000 - 200))
        reads.append(W.mutate(rng, genome[st + 20: st + 20 + n], 0.04, 0.03))
        starts.append(st)
    reads = [x if len(x) else np.zeros(1, np.uint8) for x in reads]
    qs = W.SeqSet.from_list(reads)
    pairs = np.zeros(qs.n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.arange(qs.n)
    pairs["t_offset"] = starts
    pairs["t_len"] = 80 if uniform else 60 + rng.integers(0, 140, qs.n)
    S = W.dna_matrix(1, -4)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, 6, 1, mode=mode, free_ends=fe, pairs=pairs)
    ctx.traceback(r)
    h = r.hits()
    check_traceback(h, r.cigar(), qs, db, S, 6, 1, mode, fe)
    assert (h["flags"] & dsa.HIT_HAS_TRACEBACK).sum() >= len(h) // 2


@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 9)])
def test_packed_pairs_small_alphabet_asymmetric(ctx, mode, fe):
    """Byte-permute substitution form: 3-letter alphabet, asymmetric matrix with
    negative S + o entries (sign extension of each half), odd pair count."""
    rng = np.random.default_rng(610 + mode)
    S = np.array([[3, -4, 1], [-2, 2, -6], [0, -5, 4]], dtype=np.int8)
    qs = W.SeqSet.from_list([rng.integers(0, 3, n).astype(np.uint8) for n in rng.integers(1, 90, 40)])
    db = W.SeqSet.from_list([rng.integers(0, 3, n).astype(np.uint8) for n in rng.integers(1, 300, 30)])
    pairs = _pairs_case(rng, qs, db, 333)
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, 4, 1, mode, fe, pair_toff=pairs["t_offset"],
                                    pair_tlen=pairs["t_len"])
    d = ctx.load_set(db, 3)
    q = ctx.load_set(qs, 3)
    r = ctx.align(d, q, S, 4, 1, mode=mode, free_ends=fe, pairs=pairs)
    ctx.sync()
    h = r.hits()
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"3-letter pairs mode={mode}")
    assert r.phase_cells()["inter16"] > 0


@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 12)])
@pytest.mark.parametrize("case", ["protein", "dna_wide_open"])
def test_thread_traceback_shared_table_form(ctx, case, mode, fe, monkeypatch):
    """The thread-per-hit traceback's shared-memory substitution form (more
    than 4 letters, or S + o outside int8 so the byte tables cannot hold it)
    against the oracle, forced onto the thread path."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1")
    rng = np.random.default_rng(77 + mode + fe + (0 if case == "protein" else 1000))
    if case == "protein":
        bg = W.protein_background()
        base = [rng.choice(20, int(n), p=bg).astype(np.uint8) for n in rng.integers(20, 200, 6)]
        targets = [W.mutate(rng, base[k % 6], 0.15, 0.04, alphabet=20) for k in range(30)]
        S, o, e, A = W.blosum62(), 11, 1, 24
    else:
        base = [rng.integers(0, 4, int(n)).astype(np.uint8) for n in rng.integers(20, 200, 6)]
        targets = [W.mutate(rng, base[k % 6], 0.05, 0.02) for k in range(30)]
        S, o, e, A = W.dna_matrix(5, -4), 125, 3, 4    # S + o up to 130
    targets = [t if len(t) else np.zeros(1, np.uint8) for t in targets]
    qs = W.SeqSet.from_list(base)
    db = W.SeqSet.from_list(targets)
    d = ctx.load_set(db, A)
    q = ctx.load_set(qs, A)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe)
    ctx.traceback(r)
    check_traceback(r.hits(), r.cigar(), qs, db, S, o, e, mode, fe)


BAND_PARAMS = [
    ("dna_1_-4_6_1", W.dna_matrix(1, -4), 6, 1),
    ("o_eq_e", W.dna_matrix(2, -3), 3, 3),
    ("e_zero", W.dna_matrix(2, -3), 4, 0),
    ("smax_zero", np.array([[0, -3, -3, -3], [-3, 0, -3, -3], [-3, -3, 0, -3], [-3, -3, -3, 0]], np.int8), 2, 1),
    ("smax_neg", np.array([[-1, -4, -4, -4], [-4, -1, -4, -4], [-4, -4, -1, -4], [-4, -4, -4, -1]], np.int8), 2, 1),
    ("big_match", W.dna_matrix(9, -2), 10, 1),
]


@pytest.mark.parametrize("name,S,o,e", BAND_PARAMS, ids=[p[0] for p in BAND_PARAMS])
@pytest.mark.parametrize("mode,fe", [(dsa.SEMIGLOBAL, 12), (dsa.GLOBAL, 15), (dsa.LOCAL, 15),
                                     (dsa.SEMIGLOBAL, 3)])
def test_traceback_band_parameter_sweep(ctx, name, S, o, e, mode, fe, monkeypatch):
    """Score-derived traceback windows under unusual scoring (no extension
    penalty, o = e, largest entry 0 or negative, large matches) and heavy
    indels: thread-per-hit path against the oracle's full-rectangle walk."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1")
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 1000 + 7 * mode + fe)
    genome = rng.integers(0, 4, 8000).astype(np.uint8)
    db = W.SeqSet.from_list([genome])
    reads, starts = [], []
    for n in rng.integers(5, 60, 120):
        st = int(rng.integers(0, 8000 - 150))
        reads.append(W.mutate(rng, genome[st + 15: st + 15 + n], 0.06, 0.08))
        starts.append(st)
    reads = [x if len(x) else np.zeros(1, np.uint8) for x in reads]
    qs = W.SeqSet.from_list(reads)
    pairs = np.zeros(qs.n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.arange(qs.n)
    pairs["t_offset"] = starts
    pairs["t_len"] = 40 + rng.integers(0, 100, qs.n)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, pairs=pairs)
    ctx.traceback(r)
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, o, e, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"band sweep {name}")
    check_traceback(h, r.cigar(), qs, db, S, o, e, mode, fe)


@pytest.mark.parametrize("name,S,o,e", BAND_PARAMS[:4], ids=[p[0] for p in BAND_PARAMS[:4]])
@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.LOCAL, 15)])
def test_long_pair_band_parameter_sweep(ctx, name, S, o, e, mode, fe):
    """The same scoring corner cases on pairs above the long-pair threshold."""
    rng = np.random.default_rng(zlib.crc32(name.encode()) % 1000 + 31 * mode)
    a = rng.integers(0, 4, 2300).astype(np.uint8)
    qs = W.SeqSet.from_list([a, rng.integers(0, 4, 2100).astype(np.uint8)])
    db = W.SeqSet.from_list([W.mutate(rng, a, 0.04, 0.03), rng.integers(0, 4, 2050).astype(np.uint8)])
    pairs = np.zeros(2, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = [0, 1]
    pairs["target_id"] = [0, 1]
    pairs["t_len"] = db.lengths
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, pairs=pairs)
    ctx.traceback(r)
    h = r.hits()
    sc, qe, te = oracle.score_pairs(qs.codes, qs.offsets, db.codes, db.offsets, pairs["query_id"],
                                    pairs["target_id"], S, o, e, mode, fe,
                                    pair_toff=pairs["t_offset"], pair_tlen=pairs["t_len"])
    assert_same((h["score"], h["q_end"], h["t_end"]), (sc, qe, te), f"long band sweep {name}")
    assert r.phase_cells()["intra16"] > 0
    check_traceback(h, r.cigar(), qs, db, S, o, e, mode, fe)


@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15)])
def test_big_all_vs_all_hits_checkpointed_traceback(ctx, mode, fe):
    """All-vs-all hits of 4 M cells or more: a checkpointed score pass over each
    hit's rectangle, then the parallel band traceback (no checkpoints from the
    search itself)."""
    rng = np.random.default_rng(900 + mode * 16 + fe)
    if mode == dsa.LOCAL:
        bg = W.protein_background()
        q0 = rng.choice(20, 2600, p=bg).astype(np.uint8)
        targets = [W.mutate(rng, q0, 0.15, 0.02, alphabet=20) for _ in range(3)]
        targets += [rng.choice(20, n, p=bg).astype(np.uint8) for n in rng.integers(50, 3000, 40)]
        queries = W.SeqSet.from_list([q0, rng.choice(20, 300, p=bg).astype(np.uint8)])
        S, o, e, A, top_k = W.blosum62(), 11, 1, 24, 5
    else:
        S, o, e, A, top_k = W.dna_matrix(2, -3), 5, 2, 4, 0
        q0 = rng.integers(0, 4, 2400).astype(np.uint8)
        targets = [W.mutate(rng, q0, 0.05, 0.01), rng.integers(0, 4, 2200).astype(np.uint8),
                   rng.integers(0, 4, 300).astype(np.uint8)]
        queries = W.SeqSet.from_list([q0, rng.integers(0, 4, 1900).astype(np.uint8)])
    db = W.SeqSet.from_list(targets)
    d = ctx.load_set(db, A)
    q = ctx.load_set(queries, A)
    r = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, top_k=top_k)
    ctx.traceback(r)
    h = r.hits()
    big = (h["q_end"].astype(np.int64) + 1) * (h["t_end"].astype(np.int64) + 1) >= (1 << 22)
    assert big.any()
    check_traceback(h, r.cigar(), queries, db, S, o, e, mode, fe)


def test_autotuned_long_threshold(ctx, tmp_path, monkeypatch):
    """The packed path's long-target threshold is tuned on the first call of a
    workload shape, stored in the cache file and reused; results stay exact."""
    cache = tmp_path / "autotune.json"
    monkeypatch.setenv("DSA_AUTOTUNE_CACHE", str(cache))
    monkeypatch.delenv("DSA_LONG_THRESHOLD", raising=False)
    rng = np.random.default_rng(77)
    bg = W.protein_background()
    queries = W.SeqSet.from_list([rng.choice(20, n, p=bg).astype(np.uint8) for n in (90, 140, 300)])
    db = W.SeqSet.from_list([rng.choice(20, n, p=bg).astype(np.uint8)
                             for n in np.concatenate([rng.integers(20, 400, 300), [5000, 9000, 20000]])])
    S = W.blosum62()
    sc, qe, te = oracle.score_all_vs_all(queries, db, S, 11, 1, oracle.LOCAL, 15)
    d = ctx.load_set(db, 24)
    q = ctx.load_set(queries, 24)
    for mode in ("retune", "cache", "off"):
        monkeypatch.setenv("DSA_AUTOTUNE", mode)
        before = ctx.kernel_launches()
        r = ctx.align(d, q, S, 11, 1)
        ctx.sync()
        launches = ctx.kernel_launches() - before
        h = r.hits()
        assert_same((h["score"], h["q_end"], h["t_end"]),
                    (sc.reshape(-1), qe.reshape(-1), te.reshape(-1)), f"autotune {mode}")
        if mode == "retune":
            tuned_launches = launches
            text = cache.read_text()
            assert "|A24|" in text and ":" in text
        elif mode == "cache":
            assert launches < tuned_launches   # no tuning passes on a cache hit
        r.free()



def test_device_staged_traceback_twice_and_fallback(ctx, monkeypatch):
    """Device staging: a second traceback call leaves traced hits alone (their
    CIGAR offsets stay valid); a result with a hit too big for the thread path
    falls back to the host staging."""
    monkeypatch.setenv("DSA_TB_THREAD_MIN", "1")
    monkeypatch.delenv("DSA_TB_HOST_STAGING", raising=False)
    rng = np.random.default_rng(5)
    genome = rng.integers(0, 4, 30000).astype(np.uint8)
    db = W.SeqSet.from_list([genome])
    reads, starts = [], []
    for n in rng.integers(20, 90, 64):
        st = int(rng.integers(0, 30000 - 3000))
        reads.append(W.mutate(rng, genome[st + 10: st + 10 + n], 0.03, 0.02))
        starts.append(st)
    reads.append(genome[100:2200].copy())   # 2,100 x 2,200 cells: above the thread path's bound
    starts.append(90)
    qs = W.SeqSet.from_list([x if len(x) else np.zeros(1, np.uint8) for x in reads])
    pairs = np.zeros(qs.n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = np.arange(qs.n)
    pairs["t_offset"] = starts
    pairs["t_len"] = 150
    pairs["t_len"][-1] = 2200
    S = W.dna_matrix(1, -4)
    d = ctx.load_set(db, 4)
    q = ctx.load_set(qs, 4)
    for with_big in (False, True):
        p = pairs if with_big else pairs[:-1]
        r = ctx.align(d, q, S, 6, 1, mode=dsa.SEMIGLOBAL, free_ends=12, pairs=p)
        ctx.traceback(r)
        first = r.hits().copy()
        ctx.traceback(r)   # nothing left to trace: unchanged
        h = r.hits()
        assert (h["cigar_off"] == first["cigar_off"]).all()
        check_traceback(h, r.cigar(), qs, db, S, 6, 1, dsa.SEMIGLOBAL, 12)
        r.free()
