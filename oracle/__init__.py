"""CPU oracle for Gotoh affine-gap alignment -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it and shares no
code with it.  See ``dsa_oracle.c`` for the recurrences and readings.
"""
from .oracle import (build, score, score_pssm, traceback, score_pairs, score_all_vs_all,  # noqa: F401
                     LOCAL, GLOBAL, SEMIGLOBAL, FREE_Q_BEGIN, FREE_Q_END, FREE_T_BEGIN,
                     FREE_T_END, OP_M, OP_I, OP_D, cigar_string, rescore_cigar)
