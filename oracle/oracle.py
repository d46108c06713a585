"""ctypes binding of the C oracle (``dsa_oracle.c``) -- test infrastructure only.

The shared library is compiled from source with the host C compiler on first
use (plain ``-O2``, no intrinsics), so it builds identically on x86_64 and
aarch64 hosts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

LOCAL, GLOBAL, SEMIGLOBAL = 0, 1, 2
FREE_Q_BEGIN, FREE_Q_END, FREE_T_BEGIN, FREE_T_END = 1, 2, 4, 8
OP_M, OP_I, OP_D = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dsa_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

_u8p = ctypes.POINTER(ctypes.c_uint8)
_i8p = ctypes.POINTER(ctypes.c_int8)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile liboracle.so if missing or older than its source; return its path.

    ``DSA_ORACLE_LIB`` names a prebuilt library to load instead (the mutation
    tests point it at deliberately broken copies)."""
    override = os.environ.get("DSA_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_score.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, _i8p,
                                         ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int, ctypes.c_uint32, _i32p, _i32p, _i32p]
            lib.oracle_traceback.argtypes = [_u8p, ctypes.c_int64, _u8p, ctypes.c_int64, _i8p,
                                             ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_int, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_int32, _i32p, _i32p, _u32p,
                                             ctypes.c_int64, _i64p]
            lib.oracle_score_pairs.argtypes = [_u8p, _u64p, _u8p, _u64p, _u32p, _u32p, _u64p,
                                               _u32p, ctypes.c_int64, _i8p, ctypes.c_int,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                               ctypes.c_uint32, ctypes.c_int, _i32p, _i32p,
                                               _i32p]
            lib.oracle_score_pssm.argtypes = [_i8p, ctypes.c_int64, _u8p, ctypes.c_int64,
                                              ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int, ctypes.c_uint32, _i32p, _i32p, _i32p]
            lib.oracle_score_pairs_pssm.argtypes = [_u8p, _u64p, _u8p, _u64p, _u32p, _u32p,
                                                    _u64p, _u32p, ctypes.c_int64, _i8p, _i8p,
                                                    ctypes.c_int, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_int, ctypes.c_uint32, ctypes.c_int,
                                                    _i32p, _i32p, _i32p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _u8(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.uint8))


def _mat(S) -> np.ndarray:
    S = np.ascontiguousarray(np.asarray(S, dtype=np.int8))
    assert S.ndim == 2 and S.shape[0] == S.shape[1]
    return S


def score(q, t, S, gap_open: int, gap_extend: int, mode: int = LOCAL, free_ends: int = 15):
    """(score, q_end, t_end) of one pair; ends are 0-based inclusive (-1: none)."""
    lib = _load()
    q = _u8(q); t = _u8(t); S = _mat(S)
    sc = ctypes.c_int32(); qe = ctypes.c_int32(); te = ctypes.c_int32()
    rc = lib.oracle_score(_p(q, _u8p), len(q), _p(t, _u8p), len(t), _p(S, _i8p), S.shape[0],
                          gap_open, gap_extend, mode, free_ends,
                          ctypes.byref(sc), ctypes.byref(qe), ctypes.byref(te))
    if rc:
        raise ValueError(f"oracle_score failed ({rc})")
    return int(sc.value), int(qe.value), int(te.value)


def traceback(q, t, S, gap_open: int, gap_extend: int, mode: int, free_ends: int,
              q_end: int, t_end: int):
    """(q_begin, t_begin, cigar) with cigar a uint32 array of (len << 4 | op)."""
    lib = _load()
    q = _u8(q); t = _u8(t); S = _mat(S)
    cap = len(q) + len(t) + 2
    cig = np.zeros(cap, dtype=np.uint32)
    qb = ctypes.c_int32(); tb = ctypes.c_int32(); nops = ctypes.c_int64()
    rc = lib.oracle_traceback(_p(q, _u8p), len(q), _p(t, _u8p), len(t), _p(S, _i8p),
                              S.shape[0], gap_open, gap_extend, mode, free_ends, q_end, t_end,
                              ctypes.byref(qb), ctypes.byref(tb), _p(cig, _u32p), cap,
                              ctypes.byref(nops))
    if rc:
        raise ValueError(f"oracle_traceback failed ({rc})")
    return int(qb.value), int(tb.value), cig[:nops.value].copy()


def score_pssm(P, t, gap_open: int, gap_extend: int, mode: int = LOCAL, free_ends: int = 15):
    """(score, q_end, t_end) of a query given as a position-specific profile:
    P is an (m, A) int8 array, P[i, a] the score of query position i against
    target residue a (Sec. II.C.2's user-defined scoring)."""
    lib = _load()
    P = np.ascontiguousarray(np.asarray(P, dtype=np.int8))
    assert P.ndim == 2
    t = _u8(t)
    sc = ctypes.c_int32(); qe = ctypes.c_int32(); te = ctypes.c_int32()
    rc = lib.oracle_score_pssm(_p(P, _i8p), P.shape[0], _p(t, _u8p), len(t), P.shape[1],
                               gap_open, gap_extend, mode, free_ends,
                               ctypes.byref(sc), ctypes.byref(qe), ctypes.byref(te))
    if rc:
        raise ValueError(f"oracle_score_pssm failed ({rc})")
    return int(sc.value), int(qe.value), int(te.value)


def score_pairs(q_codes, q_off, t_codes, t_off, pair_q, pair_t, S, gap_open, gap_extend,
                mode=LOCAL, free_ends=15, pair_toff=None, pair_tlen=None, threads=None,
                pssm=None):
    """Score many (query, target) pairs on host threads.  Returns (score, q_end, t_end).

    With ``pssm`` (an (total query residues, A) int8 array, one row per query
    residue in q_codes order) the queries are position-specific profiles and
    ``S`` only gives the alphabet size A."""
    lib = _load()
    q_codes = _u8(q_codes); t_codes = _u8(t_codes); S = _mat(S)
    q_off = np.ascontiguousarray(q_off, dtype=np.uint64)
    t_off = np.ascontiguousarray(t_off, dtype=np.uint64)
    pair_q = np.ascontiguousarray(pair_q, dtype=np.uint32)
    pair_t = np.ascontiguousarray(pair_t, dtype=np.uint32)
    n = len(pair_q)
    sc = np.zeros(n, np.int32); qe = np.zeros(n, np.int32); te = np.zeros(n, np.int32)
    if pair_toff is not None:
        pair_toff = np.ascontiguousarray(pair_toff, dtype=np.uint64)
        pair_tlen = np.ascontiguousarray(pair_tlen, dtype=np.uint32)
        toff_p, tlen_p = _p(pair_toff, _u64p), _p(pair_tlen, _u32p)
    else:
        toff_p, tlen_p = None, None
    if threads is None:
        threads = os.cpu_count() or 1
    if pssm is not None:
        pssm = np.ascontiguousarray(np.asarray(pssm, dtype=np.int8))
        assert pssm.shape == (int(q_off[-1]), S.shape[0])
    rc = lib.oracle_score_pairs_pssm(_p(q_codes, _u8p), _p(q_off, _u64p), _p(t_codes, _u8p),
                                     _p(t_off, _u64p), _p(pair_q, _u32p), _p(pair_t, _u32p),
                                     toff_p, tlen_p, n, _p(S, _i8p),
                                     None if pssm is None else _p(pssm, _i8p), S.shape[0],
                                     gap_open, gap_extend, mode, free_ends, threads,
                                     _p(sc, _i32p), _p(qe, _i32p), _p(te, _i32p))
    if rc:
        raise ValueError(f"oracle_score_pairs failed ({rc})")
    return sc, qe, te


def score_all_vs_all(queries, db, S, gap_open, gap_extend, mode=LOCAL, free_ends=15,
                     targets=None, threads=None, pssm=None):
    """Score every query against every target (or the given target ids).

    ``queries``/``db`` are objects with ``codes`` and ``offsets``.  Returns
    arrays shaped (n_queries, n_targets)."""
    tids = np.arange(db.n, dtype=np.uint32) if targets is None else np.asarray(targets, np.uint32)
    nq = queries.n
    pq = np.repeat(np.arange(nq, dtype=np.uint32), len(tids))
    pt = np.tile(tids, nq)
    sc, qe, te = score_pairs(queries.codes, queries.offsets, db.codes, db.offsets, pq, pt, S,
                             gap_open, gap_extend, mode, free_ends, threads=threads, pssm=pssm)
    shape = (nq, len(tids))
    return sc.reshape(shape), qe.reshape(shape), te.reshape(shape)


_OPS = "MID"


def cigar_string(cig) -> str:
    return "".join(f"{int(w) >> 4}{_OPS[int(w) & 15]}" for w in cig)


def rescore_cigar(q, t, S, gap_open, gap_extend, q_begin, t_begin, cig) -> int:
    """Score of the alignment a CIGAR describes (gap run of k costs o + (k-1)e)."""
    S = _mat(S)
    i, j, total = q_begin, t_begin, 0
    for w in cig:
        ln, op = int(w) >> 4, int(w) & 15
        if op == OP_M:
            for _ in range(ln):
                total += int(S[q[i], t[j]]); i += 1; j += 1
        elif op == OP_I:
            total -= gap_open + (ln - 1) * gap_extend; i += ln
        else:
            total -= gap_open + (ln - 1) * gap_extend; j += ln
    return total
