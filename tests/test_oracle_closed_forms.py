"""Pin the oracle to closed forms, textbook special cases and invariants.

* global self-alignment with a diagonally dominant matrix = sum of diagonal entries, CIGAR nM
* prohibitive gaps: local score (and end cell) = best ungapped diagonal segment (Kadane)
* match 0 / mismatch -1 / o = e = 1, global = minus the Levenshtein distance (Wagner-Fischer)
* o == e: Gotoh equals the one-matrix linear-gap DP (Needleman-Wunsch / Smith-Waterman)
* invariants: local >= 0, swap symmetry, local >= semi-global(all free) >= global,
  monotone in o and e, traceback rescored equals the score
* int16-overflow-sized inputs keep the exact int32 closed form
"""
import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import workloads as W

BLOSUM = W.blosum62()


def std_protein(rng, n):
    return rng.choice(20, size=n, p=W.protein_background()).astype(np.uint8)


def test_blosum62_properties():
    S = BLOSUM.astype(int)
    assert S.shape == (24, 24) and (S == S.T).all()
    core = S[:20, :20]
    for a in range(20):
        assert core[a, a] > np.delete(core[a], a).max()
        assert core[a, a] >= 4
    # a few published entries
    L = W.PROTEIN_LETTERS
    assert S[L.index("W"), L.index("W")] == 11 and S[L.index("C"), L.index("C")] == 9
    assert S[L.index("A"), L.index("R")] == -1 and S[L.index("*"), L.index("*")] == 1


@pytest.mark.parametrize("seed", range(6))
def test_global_self_alignment(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 400))
    for S, x in ((BLOSUM, std_protein(rng, n)),
                 (W.dna_matrix(2, -3), rng.integers(0, 4, n).astype(np.uint8))):
        o = int(rng.integers(1, 12)); e = int(rng.integers(0, o + 1))
        expect = int(sum(int(S[c, c]) for c in x))
        for mode in (oracle.GLOBAL, oracle.LOCAL):
            sc, qe, te = oracle.score(x, x, S, o, e, mode)
            assert sc == expect
        sc, qe, te = oracle.score(x, x, S, o, e, oracle.GLOBAL)
        qb, tb, cig = oracle.traceback(x, x, S, o, e, oracle.GLOBAL, 15, qe, te)
        assert (qb, tb, qe, te) == (0, 0, n - 1, n - 1)
        assert oracle.cigar_string(cig) == f"{n}M"


def kadane_cells(q, t, S):
    """Best ungapped local segment score and the set of its end cells (1-based)."""
    m, n = len(q), len(t)
    best, cells = 0, []
    for d in range(-(m - 1), n):
        run = 0
        i, j = max(0, -d), max(0, -d) + d
        while i < m and j < n:
            run = max(0, run) + int(S[q[i], t[j]])
            if run > best:
                best, cells = run, [(i + 1, j + 1)]
            elif run == best and best > 0:
                cells.append((i + 1, j + 1))
            i += 1; j += 1
    return best, cells


@pytest.mark.parametrize("seed", range(8))
def test_no_gap_local_is_kadane(seed):
    rng = np.random.default_rng(100 + seed)
    q = std_protein(rng, int(rng.integers(1, 150)))
    t = std_protein(rng, int(rng.integers(1, 150)))
    best, cells = kadane_cells(q, t, BLOSUM)
    sc, qe, te = oracle.score(q, t, BLOSUM, 10_000, 10_000, oracle.LOCAL)
    assert sc == best
    if best > 0:
        i, j = min(cells, key=lambda c: (c[1], c[0]))
        assert (qe + 1, te + 1) == (i, j)


def levenshtein(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


@pytest.mark.parametrize("seed", range(8))
def test_levenshtein(seed):
    rng = np.random.default_rng(200 + seed)
    a = rng.integers(0, 4, int(rng.integers(1, 80))).astype(np.uint8)
    b = rng.integers(0, 4, int(rng.integers(1, 80))).astype(np.uint8)
    sc, _, _ = oracle.score(a, b, W.dna_matrix(0, -1), 1, 1, oracle.GLOBAL)
    assert sc == -levenshtein(list(a), list(b))


def linear_gap_dp(q, t, S, g, mode, fe):
    """One-matrix DP with linear gap g per column; returns score and end (1-based) by min (j,i)."""
    m, n = len(q), len(t)
    H = np.zeros((m + 1, n + 1), dtype=np.int64)
    free_qb = mode == 2 and fe & 1
    free_tb = mode == 2 and fe & 4
    for i in range(1, m + 1):
        H[i, 0] = 0 if (mode == 0 or free_qb) else -g * i
    for j in range(1, n + 1):
        H[0, j] = 0 if (mode == 0 or free_tb) else -g * j
    for i in range(1, m + 1):
        for j in range(1, n + 1):
            h = max(H[i - 1, j - 1] + int(S[q[i - 1], t[j - 1]]), H[i - 1, j] - g, H[i, j - 1] - g)
            H[i, j] = max(h, 0) if mode == 0 else h
    if mode == 0:
        cand = [(i, j) for i in range(1, m + 1) for j in range(1, n + 1)]
    elif mode == 1:
        cand = [(m, n)]
    else:
        cand = [(m, n)]
        if fe & 8:
            cand += [(m, j) for j in range(n + 1)]
        if fe & 2:
            cand += [(i, n) for i in range(m + 1)]
    best = max(H[c] for c in cand)
    if mode == 0 and best == 0:
        return 0, None
    end = min((c for c in cand if H[c] == best), key=lambda c: (c[1], c[0]))
    return int(best), end


@pytest.mark.parametrize("mode,fe", [(0, 15), (1, 15), (2, 15), (2, 12), (2, 3), (2, 9)])
def test_linear_gap_special_case(mode, fe):
    rng = np.random.default_rng(300 + mode * 16 + fe)
    for _ in range(15):
        A = int(rng.choice([4, 20]))
        S = BLOSUM[:20, :20] if A == 20 else rng.integers(-3, 4, (4, 4)).astype(np.int8)
        q = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        t = rng.integers(0, A, int(rng.integers(1, 40))).astype(np.uint8)
        g = int(rng.integers(1, 6))
        best, end = linear_gap_dp(q, t, S, g, mode, fe)
        sc, qe, te = oracle.score(q, t, S, g, g, mode, fe)
        assert sc == best
        if end is not None:
            assert (qe + 1, te + 1) == end


@pytest.mark.parametrize("seed", range(10))
def test_invariants(seed):
    rng = np.random.default_rng(400 + seed)
    q = std_protein(rng, int(rng.integers(1, 120)))
    t = std_protein(rng, int(rng.integers(1, 120)))
    o = int(rng.integers(1, 14)); e = int(rng.integers(0, o + 1))
    loc = oracle.score(q, t, BLOSUM, o, e, oracle.LOCAL)[0]
    sg = oracle.score(q, t, BLOSUM, o, e, oracle.SEMIGLOBAL, 15)[0]
    glo = oracle.score(q, t, BLOSUM, o, e, oracle.GLOBAL)[0]
    assert loc >= 0 and loc >= sg >= glo
    for mode in (oracle.LOCAL, oracle.GLOBAL, oracle.SEMIGLOBAL):
        # symmetric matrix: swapping query and target keeps the score
        assert oracle.score(q, t, BLOSUM, o, e, mode)[0] == oracle.score(t, q, BLOSUM, o, e, mode)[0]
        # harsher gaps never raise the score
        base = oracle.score(q, t, BLOSUM, o, e, mode)[0]
        assert oracle.score(q, t, BLOSUM, o + 1, e, mode)[0] <= base
        if e + 1 <= o:
            assert oracle.score(q, t, BLOSUM, o, e + 1, mode)[0] <= base
        # traceback rescored equals the score and spans begin..end
        sc, qe, te = oracle.score(q, t, BLOSUM, o, e, mode)
        qb, tb, cig = oracle.traceback(q, t, BLOSUM, o, e, mode, 15, qe, te)
        if mode == oracle.LOCAL and sc == 0:
            continue
        assert oracle.rescore_cigar(q, t, BLOSUM, o, e, qb, tb, cig) == sc
        nq = sum(int(w) >> 4 for w in cig if int(w) & 15 in (0, 1))
        nt = sum(int(w) >> 4 for w in cig if int(w) & 15 in (0, 2))
        assert (qb + nq - 1, tb + nt - 1) == (qe, te)
        if mode == oracle.GLOBAL:
            assert (qb, tb, qe, te) == (0, 0, len(q) - 1, len(t) - 1)


def test_scores_beyond_int16():
    """A 5,000-residue run of the letter with the largest BLOSUM62 diagonal (W, 11)."""
    w = W.PROTEIN_LETTERS.index("W")
    x = np.full(5000, w, dtype=np.uint8)
    for mode in (oracle.LOCAL, oracle.GLOBAL, oracle.SEMIGLOBAL):
        sc, qe, te = oracle.score(x, x, BLOSUM, 11, 1, mode)
        assert sc == 55_000 and (qe, te) == (4999, 4999)
    # embedded in random flanks, local still finds it exactly
    rng = np.random.default_rng(9)
    q = np.concatenate([std_protein(rng, 300), x[:3100], std_protein(rng, 200)])
    t = np.concatenate([std_protein(rng, 50), x[:3100], std_protein(rng, 90)])
    sc, qe, te = oracle.score(q, t, BLOSUM, 11, 1, oracle.LOCAL)
    assert sc >= 3100 * 11 > 32767
