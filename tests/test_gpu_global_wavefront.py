"""Global and semi-global search of long database targets on the packed
wavefront kernel (one warp per target and query pair, DNW / DSG of
Sec. II.C.2), against the oracle.

The wavefront kernel's 16-row lanes take end-anchored 32-row strips: a
query's last row is the bottom row of one lane, the rows above its first
row reproduce row 0, and a pair's two halves may differ in strip count (the
shorter half's rows past its end are never read).  The cases vary the
query length around 16, 32 and the 512-row band, pair queries of very
different lengths, run every free-end set with small and large alphabets
and gap costs from o == e to e == 0, and take both range reruns (a score
above int16 and a boundary below it) on this kernel.  DSA_LONG_THRESHOLD
moves targets between the two kernels; every split must give the same
result.
"""
import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

from test_gpu_parity import assert_same, gpu_all, oracle_all
from test_oracle_bruteforce import MODES

pytestmark = pytest.mark.gpu

GLOBAL_MODES = [m for m in MODES if m[0] != oracle.LOCAL]


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("mode,fe", GLOBAL_MODES)
@pytest.mark.parametrize("thr", ["0", "300"])
def test_protein_lengths_around_lanes_and_bands(ctx, mode, fe, thr, monkeypatch):
    """Queries of 1-700 residues (16, 32 and 512 row edges) against 120
    targets of 1-400 plus long ones; threshold 0 puts every target on the
    wavefront kernel, 300 splits them."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", thr)
    rng = np.random.default_rng(1500 + 16 * mode + fe + int(thr))
    bg = W.protein_background()
    queries = W._make_set(rng, np.array([1, 2, 15, 16, 17, 31, 32, 33, 47, 300, 511, 512, 513, 700]), bg)
    tl = np.concatenate([rng.integers(1, 400, 120), [1, 2, 31, 32, 33, 900, 1500, 2100]])
    db = W._make_set(rng, tl, bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe} thr={thr}")
    cells = g[5].phase_cells()
    assert cells["intra16"] > 0
    if thr == "0":
        assert cells["inter16"] == 0


@pytest.mark.parametrize("mode,fe", GLOBAL_MODES)
@pytest.mark.parametrize("o,e", [(5, 2), (3, 3), (1, 0), (0, 0)])
def test_dna_related_targets_and_gap_costs(ctx, mode, fe, o, e, monkeypatch):
    """Four-letter alphabet with an asymmetric matrix (many ties), targets
    mutated from the queries (alignments with gaps near both ends), queries
    paired with partners of very different strip counts."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "0")
    rng = np.random.default_rng(1600 + 16 * mode + fe + 100 * o + e)
    S = np.array([[2, -3, -1, -4], [-2, 3, -3, -1], [-1, -4, 2, -2], [-3, -1, -2, 1]], np.int8)
    queries = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8)
                                  for n in (600, 40, 530, 7, 100, 97)])
    tl = []
    for k in range(60):
        src = queries.seq(k % queries.n)
        x = W.mutate(rng, src, 0.1, 0.05) if k % 2 else rng.integers(0, 4, int(rng.integers(1, 900)))
        tl.append(np.asarray(x, np.uint8) if len(x) else np.zeros(1, np.uint8))
    db = W.SeqSet.from_list(tl)
    orc = oracle_all(queries, db, S, o, e, mode, fe)
    g = gpu_all(ctx, queries, db, S, o, e, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe} o={o} e={e}")
    assert g[5].phase_cells()["inter16"] == 0


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15), (dsa.SEMIGLOBAL, 3),
                                     (dsa.SEMIGLOBAL, 12)])
def test_upward_rerun_on_wavefront(ctx, mode, fe, monkeypatch):
    """Self-alignment of 3,500 W residues (38,500 > 32,767) flagged by the
    wavefront kernel's column test and rerun exactly."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "0")
    w = W.PROTEIN_LETTERS.index("W")
    rng = np.random.default_rng(1700)
    bg = W.protein_background()
    run = np.full(3500, w, np.uint8)
    queries = W.SeqSet.from_list([run, rng.choice(20, 300, p=bg).astype(np.uint8)])
    db = W.SeqSet.from_list([run, rng.choice(20, 400, p=bg).astype(np.uint8), run[:2990]])
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, "upward rerun")
    assert g[0][0, 0] == 3500 * 11
    assert g[4] >= 1 and (g[3][0, 0] & dsa.HIT_RERUN_INT32)
    assert not (g[3][1, 1] & dsa.HIT_RERUN_INT32)


def test_downward_rerun_on_wavefront(ctx, monkeypatch):
    """Global pairs whose boundary alone passes -2^15 (o = 40, e = 7) are
    flagged on the wavefront kernel; the short target stays packed."""
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "0")
    rng = np.random.default_rng(1710)
    S = W.dna_matrix(2, -3)
    queries = W.random_dna(rng, 3, 2500, 3000)
    db = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8) for n in (3000, 40, 2600, 5)])
    orc = oracle_all(queries, db, S, 40, 7, oracle.GLOBAL, 15)
    g = gpu_all(ctx, queries, db, S, 40, 7, mode=dsa.GLOBAL)
    assert_same(g[:3], orc, "downward rerun")
    assert (g[3][:, 0] & dsa.HIT_RERUN_INT32).all() and (g[3][:, 2] & dsa.HIT_RERUN_INT32).all()
    assert not (g[3][:, 3] & dsa.HIT_RERUN_INT32).any()


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15)])
def test_long_target_search_with_traceback(ctx, mode, fe):
    """8 queries (64-1,500) x 3,000 lognormal targets with 40 targets of
    5,000-12,000 residues under the tuner's default threshold: the dense
    matrix against the oracle on the long targets and a sample, then top-5
    with traceback."""
    import torch
    wl = W.protein_search(seed=W.SEED_BASE + 1720 + mode + fe, n_queries=8, n_targets=3000,
                          qlo=64, qhi=1500)
    rng = np.random.default_rng(1721)
    bg = W.protein_background()
    extra = W._make_set(rng, rng.integers(5000, 12000, 40), bg)
    db = W.SeqSet.from_list([wl.db.seq(k) for k in range(wl.db.n)] +
                            [extra.seq(k) for k in range(extra.n)])
    d = ctx.load_set(db, 24)
    q = ctx.load_set(wl.queries, 24)
    dense = ctx.align(d, q, wl.matrix, 11, 1, mode=mode, free_ends=fe, flags=dsa.RESULTS_ON_DEVICE)
    ctx.sync()
    assert dense.phase_cells()["intra16"] > 0
    dh = dense.device_hits().view(-1, dsa.HIT_DTYPE.itemsize)
    sample = np.unique(np.concatenate([rng.choice(wl.db.n, 200, replace=False),
                                       np.arange(wl.db.n, db.n)]))
    idx = (torch.arange(wl.queries.n, device="cuda")[:, None] * db.n
           + torch.as_tensor(sample, device="cuda")[None, :]).reshape(-1)
    got = dh.index_select(0, idx).cpu().numpy().view(dsa.HIT_DTYPE).reshape(wl.queries.n, -1)
    sc, qe, te = oracle.score_all_vs_all(wl.queries, db, wl.matrix, 11, 1, mode, fe,
                                         targets=sample)
    assert_same((got["score"], got["q_end"], got["t_end"]), (sc, qe, te), "dense sample")
    dense.free()
    r = ctx.align(d, q, wl.matrix, 11, 1, mode=mode, free_ends=fe, top_k=5)
    ctx.traceback(r)
    cig = r.cigar()
    for x in r.hits():
        qb, tb, c = oracle.traceback(wl.queries.seq(int(x["query_id"])), db.seq(int(x["target_id"])),
                                     wl.matrix, 11, 1, mode, fe, int(x["q_end"]), int(x["t_end"]))
        got_c = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb) and got_c.tolist() == c.tolist()
