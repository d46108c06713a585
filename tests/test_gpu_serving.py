"""Serving loop: continuous batching gives each request exactly the result it gets alone.

Requests mix single protein queries (searched against a protein database,
top-10 with traceback) and DNA read batches (semi-global against windows of
a genome, traceback for every read).  They are run one at a time, then all
at once through a multi-slot server that batches and overlaps them; hits and
CIGARs must be identical.  Memory-budget gating and queue limits are checked
with an artificial budget and a tiny pending limit.
"""
import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    from paper_1701_01575_gb300 import build
    build.build()
    ctx = dsa.Context(0)
    rng = np.random.default_rng(4040)
    pdb = W._make_set(rng, W.lognormal_int(rng, 300, 0.7, 3000, 6000), W.protein_background())
    genome = rng.integers(0, 4, 300_000).astype(np.uint8)
    gdb = W.SeqSet(genome, np.array([0, len(genome)], dtype=np.uint64))
    reqs = W.serving_stream(seed=77, n_requests=30, rate=1000.0, plo=20, phi=600, dlo=20, dhi=400,
                            genome=genome)
    d_p = ctx.load_set(pdb, 24)
    d_g = ctx.load_set(gdb, 4)
    yield ctx, pdb, gdb, d_p, d_g, reqs
    ctx.close()


def submit(srv, req, d_p, d_g):
    if req.kind == "protein":
        return srv.submit(d_p, req.queries.codes, req.queries.offsets, W.blosum62(), 11, 1,
                          top_k=10, traceback=True)
    return srv.submit(d_g, req.queries.codes, req.queries.offsets, W.dna_matrix(1, -4), 6, 1,
                      mode=dsa.SEMIGLOBAL, free_ends=W.FREE_T_BEGIN | W.FREE_T_END,
                      pairs=req.pairs, traceback=True)


def wait(srv, ticket):
    srv.drain()
    res, times = srv.poll(ticket)
    assert res is not None, times
    return res.hits(), res.cigar(), times


def test_results_identical_alone_and_in_the_mix(setup):
    ctx, pdb, gdb, d_p, d_g, reqs = setup
    alone = []
    srv = dsa.Server(0, n_slots=1, max_batch_queries=1, max_batch_pairs=1)
    for r in reqs:
        alone.append(wait(srv, submit(srv, r, d_p, d_g)))
    srv.close()
    assert all(a[2]["batch_requests"] == 1 for a in alone)

    srv = dsa.Server(0, n_slots=3)
    tickets = [submit(srv, r, d_p, d_g) for r in reqs]
    srv.drain()
    mixed = [srv.poll(t) for t in tickets]
    srv.close()
    assert max(t["batch_requests"] for _, t in mixed) > 1, "nothing was batched"
    for (h1, c1, _), (res, _) in zip(alone, mixed):
        h2, c2 = res.hits(), res.cigar()
        assert (h1 == h2).all()
        assert c1.tolist() == c2.tolist()


def test_protein_requests_match_oracle(setup):
    ctx, pdb, gdb, d_p, d_g, reqs = setup
    srv = dsa.Server(0, n_slots=2)
    picks = [r for r in reqs if r.kind == "protein"][:3]
    tickets = [submit(srv, r, d_p, d_g) for r in picks]
    srv.drain()
    for r, t in zip(picks, tickets):
        res, _ = srv.poll(t)
        h = res.hits()
        sc, qe, te = oracle.score_all_vs_all(r.queries, pdb, W.blosum62(), 11, 1)
        order = sorted(range(pdb.n), key=lambda x: (-sc[0, x], x))[:10]
        assert h["target_id"].tolist() == order
        assert h["score"].tolist() == [int(sc[0, x]) for x in order]
        cig = res.cigar()
        for x in h[:3]:
            qb, tb, c = oracle.traceback(r.queries.seq(0), pdb.seq(int(x["target_id"])), W.blosum62(),
                                         11, 1, oracle.LOCAL, 15, int(x["q_end"]), int(x["t_end"]))
            got = cig[int(x["cigar_off"]):int(x["cigar_off"]) + int(x["cigar_len"])]
            assert (int(x["q_begin"]), int(x["t_begin"])) == (qb, tb) and got.tolist() == c.tolist()
    srv.close()


def test_memory_budget_gates_admission(setup):
    ctx, pdb, gdb, d_p, d_g, reqs = setup
    # a budget that holds one protein batch at a time, not two
    srv = dsa.Server(0, n_slots=3, max_batch_queries=1, mem_budget=300 << 20)
    picks = [r for r in reqs if r.kind == "protein"][:4]
    tickets = [submit(srv, r, d_p, d_g) for r in picks]
    srv.drain()
    times = [srv.poll(t)[1] for t in tickets]
    srv.close()
    spans = sorted((t["admit"], t["finish"]) for t in times)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0 - 1e-6, "two batches ran at once despite the budget"
    # a request that cannot fit at all fails with OVER_BUDGET instead of waiting forever
    srv = dsa.Server(0, n_slots=1, mem_budget=1 << 20)
    t = submit(srv, picks[0], d_p, d_g)
    srv.drain()
    res, tm = srv.poll(t)
    assert res is None and tm["status"] == dsa.ERR_OVER_BUDGET
    srv.close()


def test_pending_limit_returns_busy(setup):
    ctx, pdb, gdb, d_p, d_g, reqs = setup
    srv = dsa.Server(0, n_slots=1, max_pending=1)
    r = [x for x in reqs if x.kind == "protein"][0]
    got_busy = False
    tickets = []
    for _ in range(50):
        try:
            tickets.append(submit(srv, r, d_p, d_g))
        except dsa.DsaError as e:
            assert e.code == dsa.ERR_BUSY
            got_busy = True
            break
    srv.drain()
    srv.close()
    assert got_busy
