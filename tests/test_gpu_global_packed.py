"""Global and semi-global database search on the packed int16x2 kernel
(DNW and DSG of Sec. II.C.2), against the oracle.

The end-anchored kernel puts a query's last row at the bottom of its last
strip, so the cases below vary the query length around the strip height
(1, 27, 28, 29, 55, 56, 57 rows ... and many queries per lane stream), the
target lengths inside a warp's group (ragged tails, one-residue targets),
every free-end set, small and large alphabets with asymmetric matrices, and
the two reasons for the exact int32 rerun: a score beyond int16 (upward)
and a pair long enough for its boundary to leave the int16 range
(downward).
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


def _packed(g):
    """The score pass ran on the packed kernels (the inter-sequence kernel,
    and the wavefront kernel for the targets the tuner sends there)."""
    cells = g[5].phase_cells()
    return cells["inter16"] + cells["intra16"] > 0


@pytest.mark.parametrize("mode,fe", GLOBAL_MODES)
def test_protein_strip_boundaries(ctx, mode, fe):
    """Queries whose lengths straddle the 28-row strips; 400 targets of 1-300."""
    rng = np.random.default_rng(900 + 16 * mode + fe)
    bg = W.protein_background()
    qlens = [1, 2, 27, 28, 29, 55, 56, 57, 84, 85, 140, 203]
    queries = W._make_set(rng, qlens, bg)
    tl = rng.integers(1, 300, 400)
    tl[:5] = 1
    db = W._make_set(rng, tl, bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe}")
    assert _packed(g)


@pytest.mark.parametrize("mode,fe", GLOBAL_MODES)
@pytest.mark.parametrize("o,e", [(5, 2), (3, 3), (1, 0), (9, 1)])
def test_dna_asymmetric_and_gap_costs(ctx, mode, fe, o, e):
    """Four-letter alphabet with an asymmetric matrix (ties are frequent) and
    gap costs from o == e to e == 0; related targets so that alignments
    carry gaps."""
    rng = np.random.default_rng(930 + 16 * mode + fe + 100 * o + e)
    S = np.array([[2, -3, -1, -4], [-2, 3, -3, -1], [-1, -4, 2, -2], [-3, -1, -2, 1]], np.int8)
    base = W.random_dna(rng, 9, 1, 130)
    tl = []
    for k in range(150):
        src = base.seq(k % base.n)
        x = W.mutate(rng, src, 0.1, 0.05) if k % 2 else rng.integers(0, 4, int(rng.integers(1, 200)))
        tl.append(np.asarray(x, np.uint8) if len(x) else np.zeros(1, np.uint8))
    db = W.SeqSet.from_list(tl)
    orc = oracle_all(base, db, S, o, e, mode, fe)
    g = gpu_all(ctx, base, db, S, o, e, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe} o={o} e={e}")


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15), (dsa.SEMIGLOBAL, 5)])
def test_many_queries_per_lane_stream(ctx, mode, fe):
    """40 queries of 1-90 residues: lane streams switch queries strip by strip
    (one half starting a query while the other continues)."""
    rng = np.random.default_rng(960 + mode + fe)
    bg = W.protein_background()
    queries = W._make_set(rng, rng.integers(1, 90, 40), bg)
    db = W._make_set(rng, rng.integers(1, 120, 130), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 10, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 10, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"mode={mode} fe={fe}")


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15), (dsa.SEMIGLOBAL, 3)])
def test_upward_rerun_exact(ctx, mode, fe):
    """Self-alignment of 3,500 W residues scores 38,500 > 32,767: the running
    maximum flags the pair and the int32 rerun gives the closed form."""
    w = W.PROTEIN_LETTERS.index("W")
    rng = np.random.default_rng(970)
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


def test_downward_rerun_exact(ctx):
    """Global pairs whose boundary alone passes -2^15 (o = 40, e = 7, m + n
    beyond 4,700) are flagged and rerun; short pairs of the same search stay
    on the packed pass."""
    rng = np.random.default_rng(980)
    S = W.dna_matrix(2, -3)
    queries = W.random_dna(rng, 3, 2500, 3000)
    db = W.SeqSet.from_list([rng.integers(0, 4, n).astype(np.uint8) for n in (3000, 40, 2600, 5)])
    orc = oracle_all(queries, db, S, 40, 7, oracle.GLOBAL, 15)
    g = gpu_all(ctx, queries, db, S, 40, 7, mode=dsa.GLOBAL)
    assert_same(g[:3], orc, "downward rerun")
    assert (g[3][:, 0] & dsa.HIT_RERUN_INT32).all() and (g[3][:, 2] & dsa.HIT_RERUN_INT32).all()
    assert not (g[3][:, 3] & dsa.HIT_RERUN_INT32).any()


@pytest.mark.parametrize("mode,fe", [(dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15)])
def test_search_shape_sample_with_traceback(ctx, mode, fe):
    """8 queries (64-1,500) x 20,000 lognormal targets, top-10 with
    traceback: a sample of the dense matrix and every reported hit against
    the oracle."""
    import torch
    wl = W.protein_search(seed=W.SEED_BASE + 990 + mode + fe, n_queries=8, n_targets=20_000,
                          qlo=64, qhi=1500)
    d = ctx.load_set(wl.db, 24)
    q = ctx.load_set(wl.queries, 24)
    dense = ctx.align(d, q, wl.matrix, 11, 1, mode=mode, free_ends=fe, flags=dsa.RESULTS_ON_DEVICE)
    ctx.sync()
    dh = dense.device_hits().view(-1, dsa.HIT_DTYPE.itemsize)
    rng = np.random.default_rng(991)
    sample = np.unique(np.concatenate([rng.choice(wl.db.n, 300, replace=False),
                                       np.argsort(wl.db.lengths)[-20:]]))
    idx = (torch.arange(wl.queries.n, device="cuda")[:, None] * wl.db.n
           + torch.as_tensor(sample, device="cuda")[None, :]).reshape(-1)
    got = dh.index_select(0, idx).cpu().numpy().view(dsa.HIT_DTYPE).reshape(wl.queries.n, -1)
    sc, qe, te = oracle.score_all_vs_all(wl.queries, wl.db, wl.matrix, 11, 1, mode, fe,
                                         targets=sample)
    assert_same((got["score"], got["q_end"], got["t_end"]), (sc, qe, te), "dense sample")
    scores = dh[:, :4].contiguous().view(torch.int32).reshape(wl.queries.n, wl.db.n).cpu().numpy()
    assert _packed((None,) * 5 + (dense,))
    dense.free()
    r = ctx.align(d, q, wl.matrix, 11, 1, mode=mode, free_ends=fe, top_k=10)
    ctx.traceback(r)
    h = r.hits().reshape(wl.queries.n, 10)
    for qi in range(wl.queries.n):
        order = np.lexsort((np.arange(wl.db.n), -scores[qi]))[:10]
        assert h["target_id"][qi].tolist() == order.tolist()
    cig = r.cigar()
    for x in r.hits():
        qb, tb, c = oracle.traceback(wl.queries.seq(int(x["query_id"])), wl.db.seq(int(x["target_id"])),
                                     wl.matrix, 11, 1, mode, fe, int(x["q_end"]), int(x["t_end"]))
        got_c = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
        assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb) and got_c.tolist() == c.tolist()
