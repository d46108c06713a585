"""Seeded synthetic inputs for Gotoh alignment workloads.

This module only *draws inputs*: residue codes, lengths, offsets, substitution
matrices and gap parameters.  It contains none of the alignment arithmetic,
so both the CPU oracle (``oracle/``) and the CUDA path consume identical bytes
from here without sharing any code with each other.

The paper (Sec. II.B.1) takes three inputs: query sequences, reference
sequences and a score matrix.  Its own datasets (Table I, UniProt-derived
reference sets of 32 MB-16 GB and queries of 8-4096 residues) are not
available here, so the generators below stand in for them with the shapes of
the five workloads this library is measured on:

* ``protein_vs_db``     - one 128-residue query vs 2,000 targets, lengths U{50..500}
* ``protein_search``    - 32 queries, lengths log-uniform [64, 5000], vs 500,000 targets
                          with lognormal lengths (median 300, sigma 0.7, cap 35,000)
* ``reads_vs_windows``  - 1e6 DNA reads (150/250 bp) vs 500 bp windows of a 10 Mb genome
* ``long_pairs``        - 64 DNA pairs of 1e4..1e5 bp, second derived by mutation
* ``serving_stream``    - Poisson arrivals mixing protein queries and DNA read batches

Sequences are returned as concatenated ``uint8`` codes plus ``uint64`` offsets
(``offsets[k]..offsets[k+1]`` is sequence k), the layout the C ABI takes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 170101575

# ---------------------------------------------------------------------------
# Alphabets and substitution matrices (inputs, Sec. II.B.1: "score matrix")
# ---------------------------------------------------------------------------

PROTEIN_LETTERS = "ARNDCQEGHILKMFPSTWYVBZX*"  # NCBI BLOSUM62 row order
DNA_LETTERS = "ACGT"

# BLOSUM62 (Henikoff & Henikoff, PNAS 89:10915, 1992), in the NCBI
# distribution's row/column order including the ambiguity codes B, Z, X and
# the stop '*'.  Transcribed from the published table.
_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0 -2 -1  0 -4
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3 -1  0 -1 -4
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3  3  0 -1 -4
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3  4  1 -1 -4
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1 -3 -3 -2 -4
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2  0  3 -1 -4
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3 -1 -2 -1 -4
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3  0  0 -1 -4
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3 -3 -3 -1 -4
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1 -4 -3 -1 -4
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2  0  1 -1 -4
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1 -3 -1 -1 -4
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1 -3 -3 -1 -4
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2 -2 -1 -2 -4
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2  0  0  0 -4
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0 -1 -1  0 -4
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3 -4 -3 -2 -4
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1 -3 -2 -1 -4
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4 -3 -2 -1 -4
-2 -1  3  4 -3  0  1 -1  0 -3 -4  0 -3 -3 -2  0 -1 -4 -3 -3  4  1 -1 -4
-1  0  0  1 -3  3  4 -2  0 -3 -3  1 -1 -3 -1  0 -1 -3 -2 -2  1  4 -1 -4
 0 -1 -1 -1 -2 -1 -1 -1 -1 -1 -1 -1 -1 -1 -2  0  0 -2 -1 -1 -1 -1 -1 -4
-4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4 -4  1
"""

# Amino-acid background frequencies of Robinson & Robinson (PNAS 88:8880,
# 1991), for the 20 standard residues in PROTEIN_LETTERS order.  They only
# shape the synthetic residue distribution.
_ROBINSON_FREQ = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377,
    0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120,
    0.05841, 0.01330, 0.03216, 0.06441])


def blosum62() -> np.ndarray:
    """The 24x24 BLOSUM62 matrix as int8, row-major, PROTEIN_LETTERS order."""
    vals = [int(v) for v in _BLOSUM62_ROWS.split()]
    mat = np.array(vals, dtype=np.int8).reshape(24, 24)
    return mat


def protein_background() -> np.ndarray:
    """Background frequencies of the 20 standard residues (sum normalised to 1)."""
    return _ROBINSON_FREQ / _ROBINSON_FREQ.sum()


def dna_matrix(match: int, mismatch: int) -> np.ndarray:
    """4x4 int8 match/mismatch matrix over A,C,G,T (codes 0..3)."""
    mat = np.full((4, 4), mismatch, dtype=np.int8)
    np.fill_diagonal(mat, match)
    return mat


def encode(text: str, letters: str) -> np.ndarray:
    """Map a residue string to uint8 codes in the given alphabet order."""
    table = {c: i for i, c in enumerate(letters)}
    return np.array([table[c] for c in text.upper()], dtype=np.uint8)


def decode(codes: np.ndarray, letters: str) -> str:
    return "".join(letters[int(c)] for c in codes)


# ---------------------------------------------------------------------------
# Sequence-set container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class SeqSet:
    """Concatenated residue codes with offsets; sequence k = codes[off[k]:off[k+1]]."""
    codes: np.ndarray    # uint8
    offsets: np.ndarray  # uint64, len = n + 1

    @property
    def n(self) -> int:
        return len(self.offsets) - 1

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def seq(self, k: int) -> np.ndarray:
        return self.codes[int(self.offsets[k]):int(self.offsets[k + 1])]

    @staticmethod
    def from_list(seqs) -> "SeqSet":
        lens = np.array([len(s) for s in seqs], dtype=np.int64)
        off = np.zeros(len(seqs) + 1, dtype=np.uint64)
        off[1:] = np.cumsum(lens)
        codes = (np.concatenate([np.asarray(s, dtype=np.uint8) for s in seqs])
                 if len(seqs) else np.zeros(0, np.uint8))
        return SeqSet(codes.astype(np.uint8), off)

    def subset(self, idx) -> "SeqSet":
        return SeqSet.from_list([self.seq(int(k)) for k in idx])


def _draw_residues(rng: np.random.Generator, count: int, probs: np.ndarray,
                   chunk: int = 1 << 24) -> np.ndarray:
    """i.i.d. residue codes with the given frequencies, drawn in bounded chunks."""
    cdf = np.cumsum(probs)
    cdf[-1] = 1.0
    out = np.empty(count, dtype=np.uint8)
    for start in range(0, count, chunk):
        stop = min(count, start + chunk)
        u = rng.random(stop - start)
        out[start:stop] = np.searchsorted(cdf, u, side="right").astype(np.uint8)
    return out


def _make_set(rng, lengths: np.ndarray, probs: np.ndarray) -> SeqSet:
    lengths = np.asarray(lengths, dtype=np.int64)
    off = np.zeros(len(lengths) + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lengths)
    codes = _draw_residues(rng, int(off[-1]), probs)
    return SeqSet(codes, off)


def log_uniform_int(rng, lo: float, hi: float, size) -> np.ndarray:
    """Round(exp(U(ln lo, ln hi))), at least 1."""
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))
    return np.maximum(1, np.rint(x)).astype(np.int64)


def lognormal_int(rng, median: float, sigma: float, cap: int, size) -> np.ndarray:
    """Round(lognormal(ln median, sigma)) clamped to [1, cap]."""
    x = rng.lognormal(mean=math.log(median), sigma=sigma, size=size)
    return np.clip(np.rint(x), 1, cap).astype(np.int64)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    queries: SeqSet
    db: SeqSet
    matrix: np.ndarray          # int8 A x A, row-major
    gap_open: int
    gap_extend: int
    mode: int                   # 0 local, 1 global, 2 semi-global
    free_ends: int = 15
    pairs: Optional[np.ndarray] = None   # structured dsa_pair array, or None = all x all
    top_k: int = 0
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def alphabet_size(self) -> int:
        return int(self.matrix.shape[0])

    def cells(self) -> int:
        """Sum over aligned pairs of m * n (the DP cell count)."""
        if self.pairs is None:
            return int(self.queries.lengths.sum()) * int(self.db.lengths.sum())
        qlen = self.queries.lengths[self.pairs["query_id"].astype(np.int64)]
        return int((qlen * self.pairs["t_len"].astype(np.int64)).sum())


# Mirrors the C struct dsa_pair {uint32 query_id, target_id; uint64 t_offset; uint32 t_len; pad}.
PAIR_DTYPE = np.dtype([("query_id", "<u4"), ("target_id", "<u4"), ("t_offset", "<u8"),
                       ("t_len", "<u4"), ("_pad", "<u4")])

MODE_LOCAL, MODE_GLOBAL, MODE_SEMIGLOBAL = 0, 1, 2
FREE_Q_BEGIN, FREE_Q_END, FREE_T_BEGIN, FREE_T_END = 1, 2, 4, 8


def protein_vs_db(seed: int = SEED_BASE + 0, n_targets: int = 2000, query_len: int = 128,
                  lo: int = 50, hi: int = 500) -> Workload:
    """One protein query vs a DB with uniform target lengths; BLOSUM62 11/1, local."""
    rng = np.random.default_rng(seed)
    bg = protein_background()
    queries = _make_set(rng, np.array([query_len]), bg)
    db = _make_set(rng, rng.integers(lo, hi + 1, size=n_targets), bg)
    return Workload("protein_vs_db", queries, db, blosum62(), 11, 1, MODE_LOCAL,
                    meta=dict(seed=seed, n_targets=n_targets, query_len=query_len))


def protein_search(seed: int = SEED_BASE + 1, n_queries: int = 32, n_targets: int = 500_000,
                   qlo: int = 64, qhi: int = 5000, median: float = 300.0,
                   sigma: float = 0.7, cap: int = 35_000, top_k: int = 10) -> Workload:
    """Batched protein DB search: log-uniform query lengths, lognormal DB lengths."""
    rng = np.random.default_rng(seed)
    bg = protein_background()
    queries = _make_set(rng, log_uniform_int(rng, qlo, qhi, n_queries), bg)
    db = _make_set(rng, lognormal_int(rng, median, sigma, cap, n_targets), bg)
    return Workload("protein_search", queries, db, blosum62(), 11, 1, MODE_LOCAL,
                    top_k=top_k, meta=dict(seed=seed, n_queries=n_queries, n_targets=n_targets))


def _geometric_len(rng) -> int:
    return int(rng.geometric(0.5))


def _apply_events(rng, src: np.ndarray, positions, out_len: Optional[int], alphabet: int):
    """Indels at the given source positions (insertion or deletion with equal
    odds, length geometric p=0.5 on {1,2,...}); stops after out_len residues."""
    n = len(src)
    pos = 0
    pieces = []
    emitted = 0
    for p in positions:
        if p < pos:
            continue
        if out_len is not None and emitted + (p - pos) >= out_len:
            break
        pieces.append(src[pos:p])
        emitted += p - pos
        pos = p
        k = _geometric_len(rng)
        if rng.random() < 0.5:  # insertion of k random residues
            pieces.append(rng.integers(0, alphabet, size=k).astype(np.uint8))
            emitted += k
        else:                   # deletion of k source residues
            pos = min(n, pos + k)
    pieces.append(src[pos:])
    out = np.concatenate(pieces) if pieces else np.zeros(0, np.uint8)
    if out_len is not None:
        out = out[:out_len]
    return out.copy()


def _substitute(rng, out: np.ndarray, sub_rate: float, alphabet: int) -> np.ndarray:
    subs = np.flatnonzero(rng.random(len(out)) < sub_rate)
    if len(subs):
        shift = rng.integers(1, alphabet, size=len(subs)).astype(np.uint8)
        out[subs] = (out[subs] + shift) % alphabet
    return out.astype(np.uint8)


def mutate(rng, src: np.ndarray, sub_rate: float, indel_rate: float,
           out_len: Optional[int] = None, alphabet: int = 4) -> np.ndarray:
    """Copy ``src`` with substitutions (to a different residue) and indels.

    At each source position, with probability ``indel_rate`` an indel event
    happens (insertion or deletion with equal odds, length geometric p=0.5 on
    {1,2,...}).  If ``out_len`` is given, the walk stops once that many
    residues have been emitted (``src`` must be long enough)."""
    ev = np.flatnonzero(rng.random(len(src)) < indel_rate)
    out = _apply_events(rng, src, ev, out_len, alphabet)
    return _substitute(rng, out, sub_rate, alphabet)


def _sample_reads(rng, ref: np.ndarray, lens: np.ndarray, window: int, sub_rate: float,
                  indel_rate: float):
    """Reads of the given lengths sampled from `ref` (forward strand), with their
    windows.  Per read, indel events hit its source slice (length + 64 slack) at
    rate `indel_rate`; reads without events are the slice with substitutions,
    built in bulk.  Returns (SeqSet, pairs, origins, clean): clean[k] is True
    when read k is its source slice unchanged (no indel event in the slice
    and no substitution)."""
    n_reads = len(lens)
    ref_len = len(ref)
    slack = 64
    origins = rng.integers(0, ref_len - lens - slack, size=n_reads)
    n_events = rng.binomial(lens + slack, indel_rate)
    off = np.zeros(n_reads + 1, dtype=np.uint64)
    off[1:] = np.cumsum(lens)
    codes = np.empty(int(off[-1]), dtype=np.uint8)
    clean = np.zeros(n_reads, dtype=bool)
    for L in np.unique(lens):
        idx = np.flatnonzero((lens == L) & (n_events == 0))
        if len(idx) == 0:
            continue
        block = ref[origins[idx][:, None] + np.arange(L)[None, :]]
        hit = rng.random(block.shape) < sub_rate
        clean[idx] = ~hit.any(axis=1)
        shift = rng.integers(1, 4, size=int(hit.sum())).astype(np.uint8)
        block[hit] = (block[hit] + shift) % 4
        codes[off[idx].astype(np.int64)[:, None] + np.arange(L)[None, :]] = block
    for k in np.flatnonzero(n_events > 0):
        L = int(lens[k]); o = int(origins[k])
        src = ref[o:o + L + slack]
        ev = np.sort(rng.choice(L + slack, size=int(n_events[k]), replace=False))
        r = _substitute(rng, _apply_events(rng, src, ev, L, 4), sub_rate, 4)
        codes[int(off[k]):int(off[k]) + L] = r
    queries = SeqSet(codes, off)
    pairs = np.zeros(n_reads, dtype=PAIR_DTYPE)
    pairs["query_id"] = np.arange(n_reads, dtype=np.uint32)
    pairs["target_id"] = 0
    start = origins + (lens - window) // 2   # window centred on the read's span
    start = np.clip(start, 0, ref_len - window)
    pairs["t_offset"] = start.astype(np.uint64)
    pairs["t_len"] = window
    return queries, pairs, origins, clean


def reads_vs_windows(seed: int = SEED_BASE + 2, n_reads: int = 1_000_000,
                     ref_len: int = 10_000_000, read_lens=(150, 250), window: int = 500,
                     sub_rate: float = 0.01, indel_rate: float = 0.001) -> Workload:
    """DNA reads sampled from a random genome, each paired with a window around its origin.

    The DB is the genome (one sequence); ``pairs`` holds one (read, window) pair per
    read with ``t_offset`` = window start.  Semi-global with free target ends."""
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 4, size=ref_len).astype(np.uint8)
    lens = np.where(np.arange(n_reads) < n_reads // 2, read_lens[0], read_lens[1]).astype(np.int64)
    rng.shuffle(lens)
    queries, pairs, origins, clean = _sample_reads(rng, ref, lens, window, sub_rate, indel_rate)
    db = SeqSet(ref, np.array([0, ref_len], dtype=np.uint64))
    return Workload("reads_vs_windows", queries, db, dna_matrix(1, -4), 6, 1, MODE_SEMIGLOBAL,
                    free_ends=FREE_T_BEGIN | FREE_T_END, pairs=pairs,
                    meta=dict(seed=seed, n_reads=n_reads, ref_len=ref_len,
                              origins=origins.astype(np.int64), clean=clean))


def long_pairs(seed: int = SEED_BASE + 3, n_pairs: int = 64, lo: int = 10_000,
               hi: int = 100_000, mode: int = MODE_GLOBAL) -> Workload:
    """DNA pairs: first sequence random, second derived by 5% subs and 1% indels."""
    rng = np.random.default_rng(seed)
    lens = log_uniform_int(rng, lo, hi, n_pairs)
    firsts, seconds = [], []
    for L in lens:
        a = rng.integers(0, 4, size=int(L)).astype(np.uint8)
        b = mutate(rng, a, 0.05, 0.01)
        if len(b) == 0:
            b = a[:1].copy()
        firsts.append(a)
        seconds.append(b)
    queries = SeqSet.from_list(firsts)
    db = SeqSet.from_list(seconds)
    pairs = np.zeros(n_pairs, dtype=PAIR_DTYPE)
    pairs["query_id"] = np.arange(n_pairs, dtype=np.uint32)
    pairs["target_id"] = np.arange(n_pairs, dtype=np.uint32)
    pairs["t_offset"] = 0
    pairs["t_len"] = db.lengths.astype(np.uint32)
    return Workload("long_pairs", queries, db, dna_matrix(2, -3), 5, 2, mode, pairs=pairs,
                    meta=dict(seed=seed, n_pairs=n_pairs, lo=lo, hi=hi))


def reads_from_reference(rng, ref: np.ndarray, n_reads: int, read_len: int = 150,
                         window: int = 500, sub_rate: float = 0.01, indel_rate: float = 0.001):
    """Reads sampled from `ref` (forward strand) with their windows: (SeqSet, pairs)."""
    lens = np.full(n_reads, read_len, dtype=np.int64)
    queries, pairs, _, _ = _sample_reads(rng, ref, lens, window, sub_rate, indel_rate)
    return queries, pairs


@dataclasses.dataclass
class Request:
    kind: str               # "protein" or "dna"
    queries: SeqSet
    pairs: Optional[np.ndarray]
    arrival: float          # seconds after the stream start


def serving_stream(seed: int = SEED_BASE + 4, n_requests: int = 100, rate: float = 10.0,
                   protein_frac: float = 0.7, plo: int = 50, phi: int = 2000,
                   dlo: int = 1000, dhi: int = 100_000, genome: Optional[np.ndarray] = None):
    """Poisson arrivals (rate per second) of protein queries (log-uniform lengths,
    searched against a protein database) and DNA read batches (log-uniform counts of
    150 bp reads against 500 bp windows of `genome`)."""
    rng = np.random.default_rng(seed)
    bg = protein_background()
    t = 0.0
    out = []
    for _ in range(n_requests):
        t += float(rng.exponential(1.0 / rate))
        if rng.random() < protein_frac or genome is None:
            q = _make_set(rng, log_uniform_int(rng, plo, phi, 1), bg)
            out.append(Request("protein", q, None, t))
        else:
            n = int(log_uniform_int(rng, dlo, dhi, 1)[0])
            q, pairs = reads_from_reference(rng, genome, n)
            out.append(Request("dna", q, pairs, t))
    return out


def random_protein_pairs(rng, n: int, lo: int, hi: int) -> SeqSet:
    bg = protein_background()
    return _make_set(rng, rng.integers(lo, hi + 1, size=n), bg)


def random_dna(rng, n: int, lo: int, hi: int) -> SeqSet:
    lens = rng.integers(lo, hi + 1, size=n)
    return _make_set(rng, lens, np.full(4, 0.25))
