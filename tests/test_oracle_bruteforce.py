"""Pin the CPU oracle against exhaustive enumeration of alignments (tiny inputs).

Checks, for local, global and several semi-global free-end sets:
  * the optimal score equals the maximum over every listed alignment;
  * the reported end cell is the smallest (j, i) among optimal alignments' ends;
  * the traceback (begin, CIGAR) is one of the optimal alignments, exactly.
"""
import numpy as np
import pytest

import oracle
from bruteforce import brute, iter_small_cases, ops_from_cigar, random_matrix

MODES = [(oracle.LOCAL, 15), (oracle.GLOBAL, 15), (oracle.SEMIGLOBAL, 15),
         (oracle.SEMIGLOBAL, oracle.FREE_T_BEGIN | oracle.FREE_T_END),
         (oracle.SEMIGLOBAL, oracle.FREE_Q_BEGIN | oracle.FREE_Q_END),
         (oracle.SEMIGLOBAL, oracle.FREE_Q_BEGIN | oracle.FREE_T_END),
         (oracle.SEMIGLOBAL, 0)]


@pytest.mark.parametrize("mode,fe", MODES)
def test_oracle_matches_bruteforce(mode, fe):
    rng = np.random.default_rng(1000 + 17 * mode + fe)
    for q, t, S, o, e in iter_small_cases(rng, 120, max_len=5):
        best, end, optimal = brute(q, t, S, o, e, mode, fe)
        sc, qe, te = oracle.score(q, t, S, o, e, mode, fe)
        assert sc == best, (q, t, o, e)
        if end is None:
            assert (qe, te) == (-1, -1)
            continue
        assert (qe + 1, te + 1) == end, (q, t, S.tolist(), o, e)
        qb, tb, cig = oracle.traceback(q, t, S, o, e, mode, fe, qe, te)
        assert (qb, tb, qe + 1, te + 1, ops_from_cigar(cig)) in optimal
        assert oracle.rescore_cigar(q, t, S, o, e, qb, tb, cig) == sc


def test_oracle_matches_bruteforce_len6():
    rng = np.random.default_rng(77)
    for mode, fe in MODES[:4]:
        for q, t, S, o, e in iter_small_cases(rng, 12, alphabet_sizes=(2, 4), max_len=6):
            best, end, optimal = brute(q, t, S, o, e, mode, fe)
            sc, qe, te = oracle.score(q, t, S, o, e, mode, fe)
            assert sc == best
            if end is not None:
                assert (qe + 1, te + 1) == end
                qb, tb, cig = oracle.traceback(q, t, S, o, e, mode, fe, qe, te)
                assert (qb, tb, qe + 1, te + 1, ops_from_cigar(cig)) in optimal


@pytest.mark.parametrize("mode,fe", MODES)
def test_oracle_matches_bruteforce_len8(mode, fe):
    """Sequences of 7 and 8 residues: every alignment of every allowed pair of
    (sub)sequences enumerated (up to 265,729 op strings for 8 x 8)."""
    rng = np.random.default_rng(8000 + 17 * mode + fe)
    for k in range(5):
        A = (2, 4, 20)[k % 3]
        m, n = int(rng.integers(7, 9)), int(rng.integers(7, 9))
        q = rng.integers(0, A, m)
        t = rng.integers(0, A, n)
        S = random_matrix(rng, A)
        e = int(rng.integers(0, 4))
        o = e + int(rng.integers(0, 6))
        best, end, optimal = brute(q, t, S, o, e, mode, fe)
        sc, qe, te = oracle.score(q, t, S, o, e, mode, fe)
        assert sc == best, (q, t, S.tolist(), o, e)
        if end is None:
            assert (qe, te) == (-1, -1)
            continue
        assert (qe + 1, te + 1) == end
        qb, tb, cig = oracle.traceback(q, t, S, o, e, mode, fe, qe, te)
        assert (qb, tb, qe + 1, te + 1, ops_from_cigar(cig)) in optimal
        assert oracle.rescore_cigar(q, t, S, o, e, qb, tb, cig) == sc


def test_oracle_rejects_bad_arguments():
    S = np.eye(4, dtype=np.int8)
    q = np.zeros(3, np.uint8)
    with pytest.raises(ValueError):
        oracle.score(q, q, S, 1, 2, oracle.LOCAL)      # e > o
    with pytest.raises(ValueError):
        oracle.score(q[:0], q, S, 2, 1, oracle.LOCAL)  # empty query
    with pytest.raises(ValueError):
        oracle.score(q, q, S, 2, 1, 7)                 # bad mode
