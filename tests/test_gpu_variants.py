"""Kernel variants of the packed database search and their autotuner.

The inter-sequence kernels exist for two strip heights (28 rows, and 20 rows
that waste fewer padding rows on short queries).  Every variant must give
the oracle's scores and end cells bit for bit in every mode; the tuner
times the variants on the first call of a workload shape and records its
choice of strip height (and, in local mode, long-target threshold) in its
cache file, which the next call reads.
"""
import json

import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import dsa
from paper_1701_01575_gb300 import workloads as W

from test_gpu_parity import assert_same, gpu_all, oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1701_01575_gb300 import build
    build.build()
    c = dsa.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("rows", ["28", "20"])
@pytest.mark.parametrize("mode,fe", [(dsa.LOCAL, 15), (dsa.GLOBAL, 15), (dsa.SEMIGLOBAL, 15),
                                     (dsa.SEMIGLOBAL, 10), (dsa.SEMIGLOBAL, 5)])
def test_strip_height_variants_match_oracle(ctx, rows, mode, fe, monkeypatch):
    """Query lengths around both strip heights and many queries per lane
    stream; every target on the inter-sequence kernel."""
    monkeypatch.setenv("DSA_INTER_ROWS", rows)
    monkeypatch.setenv("DSA_LONG_THRESHOLD", "1000000")
    rng = np.random.default_rng(1200 + int(rows) + 16 * mode + fe)
    bg = W.protein_background()
    qlens = [1, 19, 20, 21, 27, 28, 29, 39, 40, 41, 56, 57, 60, 61, 140] + \
        [int(x) for x in rng.integers(1, 90, 20)]
    queries = W._make_set(rng, qlens, bg)
    db = W._make_set(rng, rng.integers(1, 260, 300), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode, fe)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode, fe=fe)
    assert_same(g[:3], orc, f"rows={rows} mode={mode} fe={fe}")
    assert g[5].phase_cells()["inter16"] > 0


@pytest.mark.parametrize("rows", ["28", "20"])
def test_strip_height_variants_saturation(ctx, rows, monkeypatch):
    """The saturation flag and int32 rerun in both variants (local)."""
    monkeypatch.setenv("DSA_INTER_ROWS", rows)
    w = W.PROTEIN_LETTERS.index("W")
    run = np.full(3100, w, np.uint8)
    rng = np.random.default_rng(1250)
    bg = W.protein_background()
    queries = W.SeqSet.from_list([run, rng.choice(20, 77, p=bg).astype(np.uint8)])
    db = W.SeqSet.from_list([run, rng.choice(20, 300, p=bg).astype(np.uint8)])
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1)
    g = gpu_all(ctx, queries, db, S, 11, 1)
    assert_same(g[:3], orc, f"rows={rows}")
    assert g[0][0, 0] == 3100 * 11 and g[4] >= 1


@pytest.mark.parametrize("mode", [dsa.LOCAL, dsa.GLOBAL])
def test_tuner_records_variant_and_reuses_it(ctx, mode, tmp_path, monkeypatch):
    cache = tmp_path / "tune.json"
    monkeypatch.setenv("DSA_AUTOTUNE_CACHE", str(cache))
    monkeypatch.setenv("DSA_AUTOTUNE", "retune")
    monkeypatch.delenv("DSA_INTER_ROWS", raising=False)
    monkeypatch.delenv("DSA_LONG_THRESHOLD", raising=False)
    rng = np.random.default_rng(1300 + mode)
    bg = W.protein_background()
    queries = W._make_set(rng, rng.integers(20, 60, 12), bg)
    db = W._make_set(rng, rng.integers(30, 400, 3000), bg)
    S = W.blosum62()
    orc = oracle_all(queries, db, S, 11, 1, mode)
    g = gpu_all(ctx, queries, db, S, 11, 1, mode=mode)
    assert_same(g[:3], orc, "tuned")
    entries = json.loads(cache.read_text())
    rows = {k: v for k, v in entries.items() if k.endswith("|rows")}
    assert len(rows) == 1 and list(rows.values())[0] in (20, 28)
    key = list(rows)[0]
    assert ("|local|" in key) == (mode == dsa.LOCAL)
    if mode == dsa.LOCAL:
        assert key[:-len("|rows")] + "|thr" in entries
    # a cached choice is reused: the next call does not tune (same result,
    # cache unchanged)
    monkeypatch.setenv("DSA_AUTOTUNE", "cache")
    before = cache.read_text()
    g2 = gpu_all(ctx, queries, db, S, 11, 1, mode=mode)
    assert_same(g2[:3], orc, "cached")
    assert cache.read_text() == before
