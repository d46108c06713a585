"""Thin ctypes binding of libdsa (include/dsa.h) -- argument marshalling only.

Every step of the alignment runs in the CUDA kernels of ``libdsa.so``; this
module only converts Python/numpy/torch arguments to the C ABI's plain
pointers and sizes.  If the library is missing, every call raises: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import weakref
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdsa.so")

# status codes (dsa.h)
OK, ERR_INVALID_ARG, ERR_OOM, ERR_OVER_BUDGET, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_BUSY, \
    ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
LOCAL, GLOBAL, SEMIGLOBAL = 0, 1, 2
FREE_Q_BEGIN, FREE_Q_END, FREE_T_BEGIN, FREE_T_END = 1, 2, 4, 8
RESULTS_ON_DEVICE, FORCE_INT32, PLAIN_FORM, PAIRS_ON_DEVICE, TIMING = 1, 2, 4, 8, 16
PHASES = ("inter16", "intra16", "int32", "hits", "traceback")
HIT_RERUN_INT32, HIT_HAS_TRACEBACK = 1, 2

HIT_DTYPE = np.dtype([("score", "<i4"), ("q_begin", "<i4"), ("q_end", "<i4"), ("t_begin", "<i4"),
                      ("t_end", "<i4"), ("query_id", "<u4"), ("target_id", "<u4"),
                      ("flags", "<u4"), ("t_offset", "<u8"), ("cigar_off", "<u8"),
                      ("cigar_len", "<u4"), ("reserved", "<u4")])
PAIR_DTYPE = np.dtype([("query_id", "<u4"), ("target_id", "<u4"), ("t_offset", "<u8"),
                       ("t_len", "<u4"), ("_pad", "<u4")])
assert HIT_DTYPE.itemsize == 56 and PAIR_DTYPE.itemsize == 24

SYMBOLS = ["dsa_create", "dsa_destroy", "dsa_last_error", "dsa_mem_in_use", "dsa_db_load",
           "dsa_db_free", "dsa_db_info", "dsa_align", "dsa_align_batch", "dsa_traceback",
           "dsa_res_get", "dsa_res_stats", "dsa_res_free", "dsa_sync", "dsa_probe_issue_rate",
           "dsa_res_timing", "dsa_kernel_launches", "dsa_score_pairs_noalloc",
           "dsa_res_phase_cells", "dsa_server_create", "dsa_submit", "dsa_poll",
           "dsa_server_drain", "dsa_server_now", "dsa_server_destroy",
           "dsa_selftest_wait_timeout", "dsa_reader_open", "dsa_reader_open_mem",
           "dsa_reader_next", "dsa_reader_close", "dsa_seqs_get", "dsa_seqs_free",
           "dsa_merge_topk", "dsa_search_partitioned", "dsa_align_pssm"]
ALPHABET_DNA4, ALPHABET_DNA5, ALPHABET_PROTEIN = 1, 2, 3
READ_MAP_UNKNOWN, READ_SKIP_EMPTY = 1, 2
ALPHABET_SIZE = {ALPHABET_DNA4: 4, ALPHABET_DNA5: 5, ALPHABET_PROTEIN: 24}
REQ_SEARCH, REQ_PAIRS = 0, 1


class _Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("db", ctypes.c_void_p), ("q_codes", ctypes.c_void_p),
                ("q_offsets", ctypes.c_void_p), ("n_queries", ctypes.c_uint32),
                ("pairs", ctypes.c_void_p), ("n_pairs", ctypes.c_uint64), ("mode", ctypes.c_int),
                ("free_ends", ctypes.c_uint32), ("matrix", ctypes.c_void_p),
                ("alphabet_size", ctypes.c_int), ("gap_open", ctypes.c_int),
                ("gap_extend", ctypes.c_int), ("top_k", ctypes.c_uint32), ("traceback", ctypes.c_int)]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("n_slots", ctypes.c_uint32), ("max_batch_queries", ctypes.c_uint32),
                ("max_batch_pairs", ctypes.c_uint64), ("mem_reserve", ctypes.c_size_t),
                ("mem_budget", ctypes.c_size_t), ("max_pending", ctypes.c_uint32)]


class _Times(ctypes.Structure):
    _fields_ = [("arrive", ctypes.c_double), ("admit", ctypes.c_double), ("finish", ctypes.c_double),
                ("batch_requests", ctypes.c_uint32), ("status", ctypes.c_int)]


class DsaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libdsa error {code}: {msg}")
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32


def load_library(path: str = LIB_PATH):
    """Load libdsa.so (built by ``paper_1701_01575_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1701_01575_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    lib.dsa_last_error.restype = ctypes.c_char_p
    lib.dsa_mem_in_use.restype = ctypes.c_size_t
    lib.dsa_mem_in_use.argtypes = [_vp]
    lib.dsa_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t, _vp]
    lib.dsa_destroy.argtypes = [_vp]
    lib.dsa_db_load.argtypes = [_vp, _vp, _vp, _u32, ctypes.c_int, ctypes.POINTER(_vp)]
    lib.dsa_db_free.argtypes = [_vp]
    lib.dsa_db_info.argtypes = [_vp, ctypes.POINTER(_u32), ctypes.POINTER(_u64),
                                ctypes.POINTER(ctypes.c_int)]
    lib.dsa_align.argtypes = [_vp, _vp, _vp, _vp, _u64, ctypes.c_int, _u32, _vp, ctypes.c_int,
                              ctypes.c_int, ctypes.c_int, _u32, _u32, ctypes.POINTER(_vp)]
    lib.dsa_align_batch.argtypes = [_vp, _vp, _vp, _vp, _u32, _vp, _u64, ctypes.c_int, _u32, _vp,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _u32, _u32,
                                    ctypes.POINTER(_vp)]
    lib.dsa_traceback.argtypes = [_vp, _vp, _vp, _u64]
    lib.dsa_res_get.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_u64),
                                ctypes.POINTER(_vp), ctypes.POINTER(_u64)]
    lib.dsa_res_stats.argtypes = [_vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]
    lib.dsa_res_free.argtypes = [_vp]
    lib.dsa_sync.argtypes = [_vp]
    lib.dsa_probe_issue_rate.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.dsa_res_timing.argtypes = [_vp, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    lib.dsa_kernel_launches.argtypes = [_vp]
    lib.dsa_res_phase_cells.argtypes = [_vp, ctypes.POINTER(_u64), ctypes.c_int]
    lib.dsa_server_create.argtypes = [ctypes.c_int, ctypes.POINTER(_ServerConfig), ctypes.POINTER(_vp)]
    lib.dsa_submit.argtypes = [_vp, ctypes.POINTER(_Request), ctypes.POINTER(_u64)]
    lib.dsa_poll.argtypes = [_vp, _u64, ctypes.POINTER(_vp), ctypes.POINTER(_Times)]
    lib.dsa_server_drain.argtypes = [_vp]
    lib.dsa_server_now.argtypes = [_vp]
    lib.dsa_server_now.restype = ctypes.c_double
    lib.dsa_server_destroy.argtypes = [_vp]
    lib.dsa_selftest_wait_timeout.argtypes = [_vp, ctypes.c_int, ctypes.c_uint64]
    lib.dsa_kernel_launches.restype = ctypes.c_uint64
    lib.dsa_score_pairs_noalloc.argtypes = [_vp, _vp, _u32, _vp, _vp, _u32, _vp, _u64, ctypes.c_int,
                                            _u32, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            _u32, _vp, _vp, _vp, _vp]
    lib.dsa_reader_open.argtypes = [ctypes.c_char_p, ctypes.c_int, _u32, _u64, ctypes.POINTER(_vp)]
    lib.dsa_reader_open_mem.argtypes = [_vp, _u64, ctypes.c_int, _u32, ctypes.POINTER(_vp)]
    lib.dsa_reader_next.argtypes = [_vp, _u64, _u32, ctypes.POINTER(_vp)]
    lib.dsa_reader_close.argtypes = [_vp]
    lib.dsa_seqs_get.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_u32),
                                 ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp)]
    lib.dsa_seqs_free.argtypes = [_vp]
    lib.dsa_align_pssm.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _u32, ctypes.c_int,
                                   ctypes.c_int, _u32, _u32, ctypes.POINTER(_vp)]
    lib.dsa_merge_topk.argtypes = [_vp, _vp, _vp, _vp, _u32, _u32, _u32, _vp, ctypes.POINTER(_u64), _vp,
                                   ctypes.POINTER(_u64)]
    lib.dsa_search_partitioned.argtypes = [_vp, _vp, _vp, _u32, ctypes.c_int, _u64, _vp, ctypes.c_int,
                                           _u32, _vp, ctypes.c_int, ctypes.c_int, _u32, ctypes.c_int,
                                           ctypes.POINTER(_vp)]
    _lib = lib
    return lib


def _check(rc: int):
    if rc != OK:
        raise DsaError(rc, _lib.dsa_last_error().decode(errors="replace"))


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Database:
    """A device-resident sequence set (database or queries)."""

    def __init__(self, ctx: "Context", handle: int):
        self.ctx, self.handle = ctx, handle
        ctx._children.add(self)
        n = _u32(); r = _u64(); a = ctypes.c_int()
        _check(_lib.dsa_db_info(handle, ctypes.byref(n), ctypes.byref(r), ctypes.byref(a)))
        self.n, self.n_res, self.alphabet_size = n.value, r.value, a.value

    def free(self):
        if self.handle and self.ctx.handle:
            _check(_lib.dsa_db_free(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Result:
    def __init__(self, ctx: "Context", handle: int, on_device: bool, keep=()):
        self.ctx, self.handle, self.on_device = ctx, handle, on_device
        self._keep = keep   # sequence sets the result refers to
        ctx._children.add(self)

    def _raw(self):
        hp = _vp(); nh = _u64(); cp = _vp(); nc = _u64()
        _check(_lib.dsa_res_get(self.handle, ctypes.byref(hp), ctypes.byref(nh), ctypes.byref(cp),
                                ctypes.byref(nc)))
        return hp.value, nh.value, cp.value, nc.value

    def hits(self) -> np.ndarray:
        """Host copy of the hits as a HIT_DTYPE structured array."""
        hp, nh, cp, nc = self._raw()
        if nh == 0:
            return np.zeros(0, HIT_DTYPE)
        if self.on_device:
            import torch
            t = self.device_hits()
            return t.cpu().numpy().view(HIT_DTYPE).copy()
        buf = (ctypes.c_uint8 * (nh * HIT_DTYPE.itemsize)).from_address(hp)
        return np.frombuffer(buf, dtype=HIT_DTYPE).copy()

    def cigar(self) -> np.ndarray:
        hp, nh, cp, nc = self._raw()
        if nc == 0:
            return np.zeros(0, np.uint32)
        if self.on_device:
            import torch
            return _device_view(cp, nc * 4).cpu().numpy().view(np.uint32).copy()
        buf = (ctypes.c_uint32 * nc).from_address(cp)
        return np.frombuffer(buf, dtype=np.uint32).copy()

    def device_hits(self):
        """The hits as a uint8 CUDA tensor viewing the result's device memory (no copy)."""
        assert self.on_device, "result was not created with RESULTS_ON_DEVICE"
        hp, nh, cp, nc = self._raw()
        return _device_view(hp, nh * HIT_DTYPE.itemsize)

    def timing(self) -> dict:
        """Per-phase device milliseconds (result made with TIMING; -1 = phase did not run)."""
        ms = (ctypes.c_double * len(PHASES))()
        _check(_lib.dsa_res_timing(self.handle, ms, len(PHASES)))
        return {name: ms[k] for k, name in enumerate(PHASES)}

    def phase_cells(self) -> dict:
        c = (_u64 * len(PHASES))()
        _check(_lib.dsa_res_phase_cells(self.handle, c, len(PHASES)))
        return {name: int(c[k]) for k, name in enumerate(PHASES)}

    def stats(self):
        cells = _u64(); rr = _u64()
        _check(_lib.dsa_res_stats(self.handle, ctypes.byref(cells), ctypes.byref(rr)))
        return cells.value, rr.value

    def free(self):
        if self.handle and self.ctx.handle:
            _check(_lib.dsa_res_free(self.handle))
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _CAI:
    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1",
                                         "data": (ptr, False), "version": 3}


def _device_view(ptr: int, nbytes: int):
    import torch
    return torch.as_tensor(_CAI(ptr, nbytes), device="cuda")


class Context:
    """A libdsa context on one CUDA device, ordering work on one stream."""

    def __init__(self, device: int = 0, mem_budget: int = 0, stream=None):
        load_library()
        h = _vp()
        sh = None
        if stream is not None:
            sh = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self._children = weakref.WeakSet()
        _check(_lib.dsa_create(ctypes.byref(h), device, mem_budget, sh))
        self.handle = h.value
        self.device = device

    def close(self):
        """Free every result and sequence set of this context, then the context."""
        if getattr(self, "handle", None):
            kids = list(self._children)
            for k in kids:
                if isinstance(k, Result):
                    k.free()
            for k in kids:
                if isinstance(k, Database):
                    k.free()
            _lib.dsa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def mem_in_use(self) -> int:
        return _lib.dsa_mem_in_use(self.handle)

    def kernel_launches(self) -> int:
        return int(_lib.dsa_kernel_launches(self.handle))

    def load(self, codes: np.ndarray, offsets: np.ndarray, alphabet_size: int) -> Database:
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        h = _vp()
        _check(_lib.dsa_db_load(self.handle, _ptr(codes) if len(codes) else None, _ptr(offsets),
                                len(offsets) - 1, alphabet_size, ctypes.byref(h)))
        return Database(self, h.value)

    def load_set(self, seqset, alphabet_size: int) -> Database:
        return self.load(seqset.codes, seqset.offsets, alphabet_size)

    @staticmethod
    def _pairs_arg(pairs):
        if pairs is None:
            return None, 0, 0, None
        if hasattr(pairs, "data_ptr"):   # torch CUDA tensor of raw dsa_pair bytes
            n = pairs.numel() * pairs.element_size() // PAIR_DTYPE.itemsize
            return pairs.data_ptr(), n, PAIRS_ON_DEVICE, pairs
        arr = np.ascontiguousarray(pairs)
        if arr.dtype != PAIR_DTYPE:
            arr = arr.astype(PAIR_DTYPE)
        return _ptr(arr), len(arr), 0, arr

    def align_pssm(self, db: Database, queries: Database, pssm: np.ndarray, gap_open: int,
                   gap_extend: int, mode: int = LOCAL, free_ends: int = 15, top_k: int = 0,
                   flags: int = 0) -> Result:
        """``dsa_align_pssm``: ``pssm`` is an (n_residues(queries), A) int8 array,
        one row per query residue in the order the queries were loaded."""
        P = np.ascontiguousarray(pssm, dtype=np.int8)
        if P.ndim != 2 or P.shape != (queries.n_res, queries.alphabet_size):
            raise ValueError(f"pssm must have shape (query residues, alphabet) = "
                             f"{(queries.n_res, queries.alphabet_size)}, not {P.shape}")
        h = _vp()
        _check(_lib.dsa_align_pssm(self.handle, db.handle, queries.handle, _ptr(P), P.shape[1], mode,
                                   free_ends, gap_open, gap_extend, top_k, flags, ctypes.byref(h)))
        return Result(self, h.value, bool(flags & RESULTS_ON_DEVICE), keep=(db, queries))

    def search_partitioned(self, codes: np.ndarray, offsets: np.ndarray, alphabet_size: int,
                           queries: Database, matrix: np.ndarray, gap_open: int, gap_extend: int,
                           top_k: int, partition_residues: int, mode: int = LOCAL,
                           free_ends: int = 15, traceback: bool = True) -> Result:
        """``dsa_search_partitioned``: a host database searched one partition at
        a time; the result is host-only."""
        codes = np.ascontiguousarray(codes, dtype=np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        mat = np.ascontiguousarray(matrix, dtype=np.int8)
        h = _vp()
        _check(_lib.dsa_search_partitioned(self.handle, _ptr(codes), _ptr(offsets), len(offsets) - 1,
                                           alphabet_size, partition_residues, queries.handle, mode,
                                           free_ends, _ptr(mat), gap_open, gap_extend, top_k,
                                           1 if traceback else 0, ctypes.byref(h)))
        return Result(self, h.value, False, keep=(queries,))

    def align(self, db: Database, queries: Database, matrix: np.ndarray, gap_open: int,
              gap_extend: int, mode: int = LOCAL, free_ends: int = 15, pairs=None, top_k: int = 0,
              flags: int = 0) -> Result:
        mat = np.ascontiguousarray(matrix, dtype=np.int8)
        pp, npairs, pflag, keep = self._pairs_arg(pairs)
        h = _vp()
        _check(_lib.dsa_align(self.handle, db.handle, queries.handle, pp, npairs, mode, free_ends,
                              _ptr(mat), mat.shape[0], gap_open, gap_extend, top_k, flags | pflag,
                              ctypes.byref(h)))
        return Result(self, h.value, bool(flags & RESULTS_ON_DEVICE), keep=(db, queries))

    def align_batch(self, db: Database, q_codes: np.ndarray, q_offsets: np.ndarray,
                    matrix: np.ndarray, gap_open: int, gap_extend: int, mode: int = LOCAL,
                    free_ends: int = 15, pairs=None, top_k: int = 0, flags: int = 0) -> Result:
        q_codes = np.ascontiguousarray(q_codes, dtype=np.uint8)
        q_offsets = np.ascontiguousarray(q_offsets, dtype=np.uint64)
        mat = np.ascontiguousarray(matrix, dtype=np.int8)
        pp, npairs, pflag, keep = self._pairs_arg(pairs)
        h = _vp()
        _check(_lib.dsa_align_batch(self.handle, db.handle, _ptr(q_codes), _ptr(q_offsets),
                                    len(q_offsets) - 1, pp, npairs, mode, free_ends, _ptr(mat),
                                    mat.shape[0], gap_open, gap_extend, top_k, flags | pflag,
                                    ctypes.byref(h)))
        return Result(self, h.value, bool(flags & RESULTS_ON_DEVICE), keep=(db,))

    def traceback(self, res: Result, which: Optional[np.ndarray] = None):
        if which is None:
            _check(_lib.dsa_traceback(self.handle, res.handle, None, 0))
        else:
            w = np.ascontiguousarray(which, dtype=np.uint64)
            _check(_lib.dsa_traceback(self.handle, res.handle, _ptr(w), len(w)))

    def sync(self):
        _check(_lib.dsa_sync(self.handle))

    def selftest_wait_timeout(self, kind: int, limit_ns: int) -> int:
        """Run the bounded-wait self-test; returns dsa_sync's status (expected ERR_DEVICE_TIMEOUT)."""
        _check(_lib.dsa_selftest_wait_timeout(self.handle, kind, limit_ns))
        return _lib.dsa_sync(self.handle)

    def probe_issue_rate(self, form: int) -> float:
        r = ctypes.c_double()
        _check(_lib.dsa_probe_issue_rate(self.handle, form, ctypes.byref(r)))
        return r.value


class HostResult:
    """A result handed out by a Server: host arrays, request-local query ids."""

    def __init__(self, handle: int):
        self.handle = handle

    def _raw(self):
        hp = _vp(); nh = _u64(); cp = _vp(); nc = _u64()
        _check(_lib.dsa_res_get(self.handle, ctypes.byref(hp), ctypes.byref(nh), ctypes.byref(cp),
                                ctypes.byref(nc)))
        return hp.value, nh.value, cp.value, nc.value

    def hits(self) -> np.ndarray:
        hp, nh, cp, nc = self._raw()
        if nh == 0:
            return np.zeros(0, HIT_DTYPE)
        buf = (ctypes.c_uint8 * (nh * HIT_DTYPE.itemsize)).from_address(hp)
        return np.frombuffer(buf, dtype=HIT_DTYPE).copy()

    def cigar(self) -> np.ndarray:
        hp, nh, cp, nc = self._raw()
        if nc == 0:
            return np.zeros(0, np.uint32)
        return np.frombuffer((ctypes.c_uint32 * nc).from_address(cp), dtype=np.uint32).copy()

    def free(self):
        if self.handle:
            _lib.dsa_res_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (dsa_server_*)."""

    def __init__(self, device: int = 0, n_slots: int = 2, max_batch_queries: int = 64,
                 max_batch_pairs: int = 2_000_000, mem_reserve: int = 0, mem_budget: int = 0,
                 max_pending: int = 0):
        load_library()
        cfg = _ServerConfig(n_slots, max_batch_queries, max_batch_pairs, mem_reserve, mem_budget,
                            max_pending)
        h = _vp()
        _check(_lib.dsa_server_create(device, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def submit(self, db: Database, q_codes, q_offsets, matrix, gap_open: int, gap_extend: int,
               mode: int = LOCAL, free_ends: int = 15, top_k: int = 0, pairs=None,
               traceback: bool = True) -> int:
        qc = np.ascontiguousarray(q_codes, dtype=np.uint8)
        qo = np.ascontiguousarray(q_offsets, dtype=np.uint64)
        mat = np.ascontiguousarray(matrix, dtype=np.int8)
        pr = None if pairs is None else np.ascontiguousarray(pairs).astype(PAIR_DTYPE)
        req = _Request(REQ_PAIRS if pr is not None else REQ_SEARCH, db.handle, _ptr(qc), _ptr(qo),
                       len(qo) - 1, _ptr(pr) if pr is not None else None,
                       len(pr) if pr is not None else 0, mode, free_ends, _ptr(mat), mat.shape[0],
                       gap_open, gap_extend, top_k, int(bool(traceback)))
        t = _u64()
        _check(_lib.dsa_submit(self.handle, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int):
        """(HostResult, times dict) when done, (None, None) while pending."""
        h = _vp()
        tm = _Times()
        rc = _lib.dsa_poll(self.handle, ticket, ctypes.byref(h), ctypes.byref(tm))
        if rc == ERR_BUSY:
            return None, None
        times = {"arrive": tm.arrive, "admit": tm.admit, "finish": tm.finish,
                 "batch_requests": tm.batch_requests, "status": tm.status}
        if rc != OK:
            return None, times
        return HostResult(h.value), times

    def drain(self):
        _check(_lib.dsa_server_drain(self.handle))

    def now(self) -> float:
        return _lib.dsa_server_now(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib.dsa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cigar_of(hit, cigar: np.ndarray) -> np.ndarray:
    off, n = int(hit["cigar_off"]), int(hit["cigar_len"])
    return cigar[off:off + n]


class Reader:
    """Streaming FASTA / FASTQ reader (``dsa_reader_*``): batches of whole
    records as (codes, offsets, names, header lines) -- the arrays
    ``Context.load`` takes.  Give ``path`` (a file, read in ``chunk_bytes``
    pieces) or ``data`` (bytes held for the reader's lifetime)."""

    def __init__(self, path=None, data=None, alphabet: int = ALPHABET_DNA4, flags: int = 0,
                 chunk_bytes: int = 0):
        if _lib is None:
            load_library()
        if (path is None) == (data is None):
            raise ValueError("give exactly one of path and data")
        self.alphabet_size = ALPHABET_SIZE.get(alphabet, 0)
        h = _vp()
        self._data = None
        if path is not None:
            _check(_lib.dsa_reader_open(os.fsencode(path), alphabet, flags, chunk_bytes, ctypes.byref(h)))
        else:
            self._data = ctypes.create_string_buffer(bytes(data), len(data))
            _check(_lib.dsa_reader_open_mem(ctypes.addressof(self._data), len(data), alphabet, flags,
                                            ctypes.byref(h)))
        self.handle = h.value

    def next_batch(self, max_residues: int = 0, max_seqs: int = 0):
        """The next batch, or None at the end of the input."""
        b = _vp()
        _check(_lib.dsa_reader_next(self.handle, max_residues, max_seqs, ctypes.byref(b)))
        if not b.value:
            return None
        try:
            c, o, n, nm, no, ln = _vp(), _vp(), _u32(), _vp(), _vp(), _vp()
            _check(_lib.dsa_seqs_get(b.value, ctypes.byref(c), ctypes.byref(o), ctypes.byref(n),
                                     ctypes.byref(nm), ctypes.byref(no), ctypes.byref(ln)))
            k = n.value
            offsets = np.ctypeslib.as_array(ctypes.cast(o, ctypes.POINTER(_u64)), (k + 1,)).copy()
            total = int(offsets[-1])
            codes = (np.ctypeslib.as_array(ctypes.cast(c, ctypes.POINTER(ctypes.c_uint8)), (total,)).copy()
                     if total else np.zeros(0, np.uint8))
            name_off = np.ctypeslib.as_array(ctypes.cast(no, ctypes.POINTER(_u64)), (k + 1,)).copy()
            raw = ctypes.string_at(nm, int(name_off[-1])) if name_off[-1] else b""
            names = [raw[name_off[x]:name_off[x + 1]].decode(errors="replace") for x in range(k)]
            lines = np.ctypeslib.as_array(ctypes.cast(ln, ctypes.POINTER(_u64)), (k,)).copy()
            return codes, offsets, names, lines
        finally:
            _lib.dsa_seqs_free(b.value)

    def batches(self, max_residues: int = 0, max_seqs: int = 0):
        """Every remaining batch under the given limits (0 = no limit)."""
        while True:
            b = self.next_batch(max_residues, max_seqs)
            if b is None:
                return
            yield b

    def __iter__(self):
        return self.batches()

    def close(self):
        if self.handle:
            _lib.dsa_reader_close(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def read_sequences(path=None, data=None, alphabet: int = ALPHABET_DNA4, flags: int = 0):
    """Whole input as one (codes, offsets, names, lines) batch."""
    with Reader(path=path, data=data, alphabet=alphabet, flags=flags) as r:
        b = r.next_batch()
        if b is None:
            return np.zeros(0, np.uint8), np.zeros(1, np.uint64), [], np.zeros(0, np.uint64)
        return b


def merge_topk(parts, target_base, n_queries: int, k: int):
    """``dsa_merge_topk`` over host arrays: ``parts`` is a list of (hits,
    cigar or None) per partition (hits as HIT_DTYPE arrays, query-major);
    returns the merged (hits, cigar) with global target ids."""
    if _lib is None:
        load_library()
    hs = [np.ascontiguousarray(h, dtype=HIT_DTYPE) for h, _ in parts]
    cs = [None if c is None else np.ascontiguousarray(c, dtype=np.uint32) for _, c in parts]
    n = len(parts)
    hp = (_vp * max(n, 1))(*[h.ctypes.data if len(h) else None for h in hs])
    cp = (_vp * max(n, 1))(*[None if c is None or not len(c) else c.ctypes.data for c in cs])
    nh = np.array([len(h) for h in hs] or [0], dtype=np.uint64)
    base = np.ascontiguousarray(target_base, dtype=np.uint32)
    out = np.zeros(max(1, n_queries * k), dtype=HIT_DTYPE)
    cig_cap = sum(int(h["cigar_len"].sum()) for h in hs)
    out_c = np.zeros(max(1, cig_cap), dtype=np.uint32)
    on, oc = _u64(), _u64()
    _check(_lib.dsa_merge_topk(hp, _ptr(nh), cp, _ptr(base), n, n_queries, k, _ptr(out),
                               ctypes.byref(on), _ptr(out_c), ctypes.byref(oc)))
    return out[:on.value].copy(), out_c[:oc.value].copy()
