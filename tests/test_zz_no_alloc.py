"""The allocation-free entry point agrees with dsa_align on explicit pairs.

dsa_score_pairs_noalloc serves callers that cannot allocate device memory
(an application that owns all device memory through its own pool, a serving
thread that may not block on the device allocator, code recording work while
allocation is not permitted): they pass device inputs and outputs they own,
and the library uses only a fixed scratch array compiled into it.  This test
calls it three times in a row through the C ABI -- semi-global reads, local
protein pairs, global DNA pairs with one-residue queries and windows, so a
call that left stale state in the shared scratch would show -- and checks
each call's scores and end cells against dsa_align's, bit-exactly.  A last
call mixes a pair whose window offset is near 2^64 among valid pairs: that
pair alone must come back as out of range (INT32_MIN, ends -2).

The file is named to be collected last, so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _dev(torch, arr):
    return torch.as_tensor(np.ascontiguousarray(arr), device="cuda")


def _case(call):
    from paper_1701_01575_gb300 import workloads as W
    if call == 0:   # semi-global reads in 500 bp windows
        wl = W.reads_vs_windows(seed=W.SEED_BASE + 200, n_reads=1500, ref_len=80_000)
        return wl.queries, wl.db, wl.pairs, wl.matrix, 6, 1, W.MODE_SEMIGLOBAL, wl.free_ends
    rng = np.random.default_rng(5150)   # local protein pairs with varied windows
    bg = W.protein_background()
    qs = W._make_set(rng, rng.integers(1, 300, 40), bg)
    db = W._make_set(rng, rng.integers(20, 900, 60), bg)
    n = 700
    pairs = np.zeros(n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = rng.integers(0, qs.n, n)
    pairs["target_id"] = rng.integers(0, db.n, n)
    tl = db.lengths[pairs["target_id"].astype(np.int64)]
    off = (rng.random(n) * (tl // 3)).astype(np.int64)
    pairs["t_offset"] = off
    pairs["t_len"] = np.maximum(1, (tl - off) - (rng.random(n) * (tl - off) // 4).astype(np.int64))
    if call == 1:
        return qs, db, pairs, W.blosum62(), 11, 1, W.MODE_LOCAL, 15
    # global DNA pairs, +2/-3, 5/2: row-0 and column-0 gap boundaries and the
    # (m, n) end cell, with one-residue queries and windows among them
    rng = np.random.default_rng(5151)
    dna = np.full(4, 0.25)
    qs = W._make_set(rng, np.concatenate([[1, 1, 2], rng.integers(1, 400, 37)]), dna)
    db = W._make_set(rng, rng.integers(1, 1200, 50), dna)
    n = 600
    pairs = np.zeros(n, dtype=W.PAIR_DTYPE)
    pairs["query_id"] = rng.integers(0, qs.n, n)
    pairs["target_id"] = rng.integers(0, db.n, n)
    tl = db.lengths[pairs["target_id"].astype(np.int64)]
    wl = np.maximum(1, (rng.random(n) * tl).astype(np.int64))
    wl[:25] = 1
    pairs["t_len"] = wl
    pairs["t_offset"] = (rng.random(n) * (tl - wl + 1)).astype(np.int64)
    return qs, db, pairs, W.dna_matrix(2, -3), 5, 2, W.MODE_GLOBAL, 15


def test_noalloc_matches_dsa_align_on_calls_in_a_row():
    import torch
    from paper_1701_01575_gb300 import build, dsa
    build.build()
    lib = dsa.load_library()
    ctx = dsa.Context(0)

    def call_noalloc(qc, qo, nq, tc, to, nt, pairs, mode, fe, dm, A, o, e):
        dp = _dev(torch, pairs.view(np.uint8))
        n = len(pairs)
        sc = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        qe = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        te = torch.full((n,), 12345, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream().cuda_stream
        rc = lib.dsa_score_pairs_noalloc(
            qc.data_ptr(), qo.data_ptr(), nq, tc.data_ptr(), to.data_ptr(), nt,
            dp.data_ptr(), n, mode, fe, dm.data_ptr(), A, o, e,
            int(min(pairs["t_len"].max(), 32768)), sc.data_ptr(), qe.data_ptr(), te.data_ptr(),
            stream)
        assert rc == 0, lib.dsa_last_error()
        torch.cuda.synchronize()
        return sc.cpu().numpy(), qe.cpu().numpy(), te.cpu().numpy()

    try:
        for call in range(3):
            qs, db, pairs, S, o, e, mode, fe = _case(call)
            A = S.shape[0]
            d = ctx.load_set(db, A)
            q = ctx.load_set(qs, A)
            ref = ctx.align(d, q, S, o, e, mode=mode, free_ends=fe, pairs=pairs).hits()

            qc = _dev(torch, qs.codes)
            qo = _dev(torch, qs.offsets.view(np.int64))
            tc = _dev(torch, db.codes)
            to = _dev(torch, db.offsets.view(np.int64))
            dm = _dev(torch, S.view(np.uint8))
            sc, qe, te = call_noalloc(qc, qo, qs.n, tc, to, db.n, pairs, mode, fe, dm, A, o, e)
            assert (sc == ref["score"]).all(), f"call {call}: scores differ"
            assert (qe == ref["q_end"]).all(), f"call {call}: q_end differs"
            assert (te == ref["t_end"]).all(), f"call {call}: t_end differs"

        # a window offset near 2^64 (t_offset + t_len wraps to 0) among valid
        # pairs: only that pair is reported out of range
        bad = pairs.copy()
        bad["t_offset"][7] = np.uint64(2**64 - 1)
        bad["t_len"][7] = 1
        sc, qe, te = call_noalloc(qc, qo, qs.n, tc, to, db.n, bad, mode, fe, dm, A, o, e)
        keep = np.arange(len(bad)) != 7
        assert (sc[7], qe[7], te[7]) == (np.iinfo(np.int32).min, -2, -2)
        assert (sc[keep] == ref["score"][keep]).all() and (qe[keep] == ref["q_end"][keep]).all()
        assert (te[keep] == ref["t_end"][keep]).all()
        n = len(pairs)
        dp = _dev(torch, pairs.view(np.uint8))
        sc = torch.zeros(n, dtype=torch.int32, device="cuda")
        qe = torch.zeros(n, dtype=torch.int32, device="cuda")
        te = torch.zeros(n, dtype=torch.int32, device="cuda")
        # sizes beyond the scratch's limit are rejected with a clear error
        rc = lib.dsa_score_pairs_noalloc(qc.data_ptr(), qo.data_ptr(), qs.n, tc.data_ptr(),
                                         to.data_ptr(), db.n, dp.data_ptr(), n, mode, fe,
                                         dm.data_ptr(), A, o, e, 1 << 20, sc.data_ptr(),
                                         qe.data_ptr(), te.data_ptr(), None)
        assert rc == dsa.ERR_INVALID_ARG and b"max_t_len" in lib.dsa_last_error()
    finally:
        ctx.close()
