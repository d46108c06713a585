"""Brute-force alignment enumeration used to pin the CPU oracle.

Every alignment between every allowed (start, end) pair of prefixes is listed
explicitly as an op string over {M, I, D} and scored by run-length gap costs
(a run of k gap columns costs o + (k-1)e).  Nothing here is a dynamic
program: the optimum is a max over an explicit list, so a dropped term, a
wrong boundary or a transposed matrix in the oracle shows up as a mismatch.

Allowed start cells (a0, b0) and end cells (i, j) (prefix lengths):
  local:       any a0 <= i, b0 <= j; the empty alignment (score 0) is allowed
  global:      (0, 0) -> (m, n)
  semi-global: start on row 0 or column 0, with a0 > 0 only if the query begin
               is free and b0 > 0 only if the target begin is free; end on row
               m or column n, with i < m only if the query end is free and
               j < n only if the target end is free.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

M, I, D = 0, 1, 2
FREE_Q_BEGIN, FREE_Q_END, FREE_T_BEGIN, FREE_T_END = 1, 2, 4, 8


@functools.lru_cache(maxsize=None)
def alignments(a: int, b: int):
    """All op strings aligning a query residues with b target residues."""
    if a == 0 and b == 0:
        return ((),)
    out = []
    if a > 0 and b > 0:
        out += [(M,) + s for s in alignments(a - 1, b - 1)]
    if a > 0:
        out += [(I,) + s for s in alignments(a - 1, b)]
    if b > 0:
        out += [(D,) + s for s in alignments(a, b - 1)]
    return tuple(out)


@functools.lru_cache(maxsize=None)
def _shape_tables(a: int, b: int):
    """Per op string over an a x b grid: the (x, y) M-column incidence, the
    number of gap runs and the total gap length (a run of k gap columns costs
    o + (k-1)e = (o - e) + k e, so the gaps of an op string cost
    runs (o - e) + length e)."""
    ops = alignments(a, b)
    inc = np.zeros((len(ops), max(1, a * b)), dtype=np.int32)
    runs = np.zeros(len(ops), dtype=np.int64)
    glen = np.zeros(len(ops), dtype=np.int64)
    for k, s in enumerate(ops):
        x = y = 0
        prev = None
        for op in s:
            if op == M:
                inc[k, x * b + y] = 1
                x += 1; y += 1
            else:
                if op == I:
                    x += 1
                else:
                    y += 1
                glen[k] += 1
                if op != prev:
                    runs[k] += 1
            prev = op
    return ops, inc, runs, glen


def _tables(a: int, b: int, o: int, e: int):
    """Op strings, M-column incidence and gap cost of every alignment of a x b."""
    ops, inc, runs, glen = _shape_tables(a, b)
    return ops, inc, runs * (o - e) + glen * e


def _allowed(m, n, mode, fe):
    """Yield allowed (a0, b0, i, j) quadruples."""
    if mode == 1:
        yield (0, 0, m, n)
        return
    for a0 in range(m + 1):
        for b0 in range(n + 1):
            if mode == 2:
                if not (a0 == 0 or b0 == 0):
                    continue
                if a0 > 0 and not (fe & FREE_Q_BEGIN):
                    continue
                if b0 > 0 and not (fe & FREE_T_BEGIN):
                    continue
            for i in range(a0, m + 1):
                for j in range(b0, n + 1):
                    if mode == 2:
                        if not (i == m or j == n):
                            continue
                        if i < m and not (fe & FREE_Q_END):
                            continue
                        if j < n and not (fe & FREE_T_END):
                            continue
                    yield (a0, b0, i, j)


def brute(q, t, S, o, e, mode, fe=15):
    """Return (best, end_cell, optimal) where end_cell = (i, j) 1-based prefix lengths
    chosen as the smallest (j, i) among optimal alignments, or None for an empty local
    optimum, and ``optimal`` is the set of (a0, b0, i, j, ops) achieving ``best``."""
    q = np.asarray(q, dtype=np.int64)
    t = np.asarray(t, dtype=np.int64)
    S = np.asarray(S, dtype=np.int64)
    m, n = len(q), len(t)
    best = None
    cands = []
    for (a0, b0, i, j) in _allowed(m, n, mode, fe):
        a, b = i - a0, j - b0
        ops, inc, gap = _tables(a, b, o, e)
        if a * b:
            sub = S[np.ix_(q[a0:i], t[b0:j])].reshape(-1).astype(np.int32)
            scores = (inc @ sub).astype(np.int64) - gap
        else:
            scores = -gap
        top = int(scores.max())
        if best is None or top > best:
            best = top
            cands = []
        if top == best:
            for k in np.flatnonzero(scores == top):
                cands.append((a0, b0, i, j, ops[int(k)]))
    if mode == 0 and best <= 0:
        return 0, None, set()
    end = min(((c[3], c[2]) for c in cands))
    return best, (end[1], end[0]), set(cands)


def ops_from_cigar(cig):
    out = []
    for w in cig:
        out += [int(w) & 15] * (int(w) >> 4)
    return tuple(out)


def random_matrix(rng, A, lo=-4, hi=5, symmetric=False):
    S = rng.integers(lo, hi + 1, size=(A, A))
    if symmetric:
        S = np.triu(S) + np.triu(S, 1).T
    return S.astype(np.int8)


def iter_small_cases(rng, count, alphabet_sizes=(2, 4, 20), max_len=5):
    """Random tiny (q, t, S, o, e) cases; S asymmetric so a transposed lookup fails."""
    from paper_1701_01575_gb300 import workloads as W
    blosum = W.blosum62()[:20, :20]
    for k in itertools.count():
        if k >= count:
            return
        A = alphabet_sizes[k % len(alphabet_sizes)]
        S = blosum if A == 20 else random_matrix(rng, A)
        m = int(rng.integers(1, max_len + 1)); n = int(rng.integers(1, max_len + 1))
        q = rng.integers(0, A, size=m).astype(np.uint8)
        t = rng.integers(0, A, size=n).astype(np.uint8)
        o = int(rng.integers(1, 7)); e = int(rng.integers(0, o + 1))
        yield q, t, S, o, e
