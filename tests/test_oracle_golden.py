"""Pin the oracle to hand-worked alignments (tests/golden/handworked.txt).

These cases fix the exact choice among equally good alignments (end-cell
tie-break and traceback priorities), which enumeration alone cannot."""
import os

import numpy as np
import pytest

import oracle
from paper_1701_01575_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handworked.txt")


def load_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = [x.strip() for x in line.split("|")]
        cases.append(dict(name=f[0], mode=int(f[1]), fe=int(f[2]), matrix=f[3], o=int(f[4]),
                          e=int(f[5]), q=f[6], t=f[7], score=int(f[8]), qb=int(f[9]),
                          tb=int(f[10]), qe=int(f[11]), te=int(f[12]), cigar=f[13]))
    return cases


def matrix_of(spec):
    if spec == "blosum62":
        return W.blosum62(), W.PROTEIN_LETTERS
    kind, a, b = spec.split(":")
    assert kind == "dna"
    return W.dna_matrix(int(a), int(b)), W.DNA_LETTERS


CASES = load_cases()


@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_handworked(c):
    S, letters = matrix_of(c["matrix"])
    q = W.encode(c["q"], letters)
    t = W.encode(c["t"], letters)
    sc, qe, te = oracle.score(q, t, S, c["o"], c["e"], c["mode"], c["fe"])
    assert (sc, qe, te) == (c["score"], c["qe"], c["te"])
    qb, tb, cig = oracle.traceback(q, t, S, c["o"], c["e"], c["mode"], c["fe"], qe, te)
    assert (qb, tb) == (c["qb"], c["tb"])
    assert oracle.cigar_string(cig) == c["cigar"]


def test_golden_file_has_cases():
    assert len(CASES) >= 10
