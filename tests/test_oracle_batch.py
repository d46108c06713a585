"""Pin the oracle's batch dispatcher (``oracle.score_pairs``, matrix form).

Every explicit-pair parity test (reads in windows, long pairs, packed pairs)
reads its expected values from this path, so it is checked against
something other than itself:

* brute force: pairs of tiny queries against tiny windows of longer targets
  (ragged query offsets, windows at the start, middle and end of a target,
  windows of one residue), scored by exhaustive enumeration of the window
  slice ``t[t_offset : t_offset + t_len]`` -- the batch must return the
  enumeration's optimum and smallest (j, i) end cell, relative to the window;
* the single-pair scorer on explicit slices, at sizes the enumeration cannot
  reach, with and without windows, in every mode and several free-end sets;
* all-vs-all dispatch (no windows) lands pair k on (pair_q[k], pair_t[k]).
"""
import numpy as np
import pytest

import oracle
from bruteforce import brute, random_matrix

from test_oracle_bruteforce import MODES


def _set(lens, A, rng):
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
    return rng.integers(0, A, int(off[-1])).astype(np.uint8), off


@pytest.mark.parametrize("mode,fe", MODES)
def test_windows_match_bruteforce(mode, fe):
    rng = np.random.default_rng(6100 + 13 * mode + fe)
    A = (2, 4, 20)[(mode + fe) % 3]
    S = random_matrix(rng, A)
    q_lens = [int(x) for x in rng.integers(1, 6, 5)]
    t_lens = [int(x) for x in rng.integers(6, 30, 3)]
    q_codes, q_off = _set(q_lens, A, rng)
    t_codes, t_off = _set(t_lens, A, rng)
    pq, pt, toff, tlen = [], [], [], []
    for k in range(60):
        qi, ti = int(rng.integers(0, 5)), int(rng.integers(0, 3))
        L = t_lens[ti]
        n = int(rng.integers(1, 6))
        where = k % 3                      # window at the start, the end, or inside
        start = 0 if where == 0 else (L - n if where == 1 else int(rng.integers(0, L - n + 1)))
        pq.append(qi); pt.append(ti); toff.append(start); tlen.append(n)
    e = int(rng.integers(0, 3)); o = e + int(rng.integers(0, 5))
    sc, qe, te = oracle.score_pairs(q_codes, q_off, t_codes, t_off, pq, pt, S, o, e, mode, fe,
                                    pair_toff=toff, pair_tlen=tlen, threads=3)
    for k in range(len(pq)):
        q = q_codes[int(q_off[pq[k]]):int(q_off[pq[k] + 1])]
        base = int(t_off[pt[k]]) + toff[k]
        w = t_codes[base:base + tlen[k]]
        best, end, _ = brute(q, w, S, o, e, mode, fe)
        assert sc[k] == best, (k, q.tolist(), w.tolist(), o, e)
        if end is None:
            assert (qe[k], te[k]) == (-1, -1)
        else:
            assert (qe[k] + 1, te[k] + 1) == end, k


@pytest.mark.parametrize("mode,fe", MODES[:5])
@pytest.mark.parametrize("windows", [False, True])
def test_batch_equals_single_pair_scorer(mode, fe, windows):
    rng = np.random.default_rng(6200 + 7 * mode + fe + (100 if windows else 0))
    A = 20 if mode == oracle.LOCAL else 4
    S = random_matrix(rng, A)
    q_lens = [int(x) for x in rng.integers(1, 120, 9)]
    t_lens = [int(x) for x in rng.integers(1, 400, 11)]
    q_codes, q_off = _set(q_lens, A, rng)
    t_codes, t_off = _set(t_lens, A, rng)
    n_pairs = 150
    pq = rng.integers(0, 9, n_pairs).astype(np.uint32)
    pt = rng.integers(0, 11, n_pairs).astype(np.uint32)
    toff = tlen = None
    if windows:
        L = np.array(t_lens)[pt]
        tlen = np.array([int(rng.integers(1, l + 1)) for l in L], dtype=np.uint32)
        toff = np.array([int(rng.integers(0, l - w + 1)) for l, w in zip(L, tlen)], dtype=np.uint64)
    sc, qe, te = oracle.score_pairs(q_codes, q_off, t_codes, t_off, pq, pt, S, 7, 2, mode, fe,
                                    pair_toff=toff, pair_tlen=tlen, threads=4)
    for k in range(n_pairs):
        q = q_codes[int(q_off[pq[k]]):int(q_off[pq[k] + 1])]
        a, b = int(t_off[pt[k]]), int(t_off[pt[k] + 1])
        if windows:
            a += int(toff[k]); b = a + int(tlen[k])
        assert (sc[k], qe[k], te[k]) == oracle.score(q, t_codes[a:b], S, 7, 2, mode, fe), k


def test_all_vs_all_lands_on_the_right_cell():
    """A query scores highest against its own copy in the database: the
    dense matrix's argmax per row must be that target (an index swap or a
    transposed reshape moves it)."""
    rng = np.random.default_rng(6300)
    A = 20
    S = np.full((A, A), -3, np.int8)
    np.fill_diagonal(S, 5)
    q_lens = [31, 7, 52, 19]
    q_codes, q_off = _set(q_lens, A, rng)

    class _S:
        def __init__(self, codes, off):
            self.codes, self.offsets, self.n = codes, off, len(off) - 1

    # database: 6 random targets, then the queries' copies at ids 6..9
    noise_codes, noise_off = _set([40] * 6, A, rng)
    db_codes = np.concatenate([noise_codes, q_codes])
    db_off = np.concatenate([noise_off, noise_off[-1] + q_off[1:]]).astype(np.uint64)
    sc, qe, te = oracle.score_all_vs_all(_S(q_codes, q_off), _S(db_codes, db_off), S, 8, 1,
                                         oracle.LOCAL, threads=2)
    assert sc.shape == (4, 10)
    for qi, m in enumerate(q_lens):
        assert int(np.argmax(sc[qi])) == 6 + qi
        assert sc[qi, 6 + qi] == 5 * m and (qe[qi, 6 + qi], te[qi, 6 + qi]) == (m - 1, m - 1)
