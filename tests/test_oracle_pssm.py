"""Pin the oracle's position-specific form (the user-defined scoring extension
of Sec. II.C.2: every query position has its own row of scores).

* Brute force: a query of m positions is the code string 0..m-1 over an
  m-letter "position alphabet" with the (m, A) profile as its matrix, so the
  exhaustive enumeration scores it as it stands (tiny inputs, every mode).
* Reduction: the profile whose row i is S[q_i] gives the matrix form's result.
* Batch indexing: row k of the set's profile belongs to query residue k.
* Closed forms: an all-ones profile.
"""
import numpy as np
import pytest

import oracle
from bruteforce import brute

from test_oracle_bruteforce import MODES


@pytest.mark.parametrize("mode,fe", MODES)
def test_pssm_matches_bruteforce(mode, fe):
    rng = np.random.default_rng(4000 + 31 * mode + fe)
    for k in range(100):
        A = (2, 4, 20)[k % 3]
        m = int(rng.integers(1, 6)); n = int(rng.integers(1, 6))
        P = rng.integers(-6, 7, size=(m, A)).astype(np.int8)
        t = rng.integers(0, A, n).astype(np.uint8)
        o = int(rng.integers(1, 7)); e = int(rng.integers(0, o + 1))
        best, end, _ = brute(np.arange(m), t, P, o, e, mode, fe)
        sc, qe, te = oracle.score_pssm(P, t, o, e, mode, fe)
        assert sc == best, (P.tolist(), t.tolist(), o, e)
        if end is None:
            assert (qe, te) == (-1, -1)
        else:
            assert (qe + 1, te + 1) == end


@pytest.mark.parametrize("mode,fe", MODES[:4])
def test_profile_of_the_matrix_is_the_matrix_form(mode, fe):
    rng = np.random.default_rng(91 + mode + fe)
    for _ in range(40):
        A = 20
        S = rng.integers(-5, 8, size=(A, A)).astype(np.int8)   # asymmetric
        q = rng.integers(0, A, int(rng.integers(1, 60))).astype(np.uint8)
        t = rng.integers(0, A, int(rng.integers(1, 60))).astype(np.uint8)
        assert oracle.score_pssm(S[q], t, 9, 2, mode, fe) == oracle.score(q, t, S, 9, 2, mode, fe)


def test_batch_rows_follow_the_query_offsets():
    rng = np.random.default_rng(5)
    A = 4
    lens = [7, 1, 12, 5]
    q_off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    P = rng.integers(-4, 5, size=(int(q_off[-1]), A)).astype(np.int8)
    tl = [9, 3, 14]
    t_off = np.concatenate([[0], np.cumsum(tl)]).astype(np.uint64)
    t_codes = rng.integers(0, A, int(t_off[-1])).astype(np.uint8)
    pq = np.repeat(np.arange(4), 3).astype(np.uint32)
    pt = np.tile(np.arange(3), 4).astype(np.uint32)
    S = np.zeros((A, A), np.int8)
    q_codes = np.zeros(int(q_off[-1]), np.uint8)
    sc, qe, te = oracle.score_pairs(q_codes, q_off, t_codes, t_off, pq, pt, S, 3, 1, oracle.LOCAL,
                                    pssm=P)
    for k in range(len(pq)):
        a, b = int(q_off[pq[k]]), int(q_off[pq[k] + 1])
        c, d = int(t_off[pt[k]]), int(t_off[pt[k] + 1])
        assert (sc[k], qe[k], te[k]) == oracle.score_pssm(P[a:b], t_codes[c:d], 3, 1, oracle.LOCAL)


@pytest.mark.parametrize("m,n", [(1, 1), (5, 9), (30, 12), (17, 17)])
def test_all_ones_profile(m, n):
    P = np.ones((m, 4), np.int8)
    t = np.zeros(n, np.uint8)
    # local: the longest diagonal run, min(m, n), ending at the first cell reaching it
    sc, qe, te = oracle.score_pssm(P, t, 5, 1, oracle.LOCAL)
    assert sc == min(m, n) and (qe, te) == (min(m, n) - 1, min(m, n) - 1)
    # global: min(m, n) matches and one gap run of |m - n| columns
    sc, _, _ = oracle.score_pssm(P, t, 5, 1, oracle.GLOBAL)
    assert sc == min(m, n) - (0 if m == n else 5 + (abs(m - n) - 1) * 1)
