"""The oracle's pins must catch plausible mistakes.

Each case below plants one mistake in a temporary copy of the oracle source
(a transposed matrix lookup, a wrong gap cost, a wrong tie-break, a wrong
boundary, a wrong traceback priority, a misplaced query slice or pair window
in the batch dispatcher), builds it, and runs the brute-force
and hand-worked pin suites against it in a child process.  Every mutant must
fail at least one pin.  Nothing here touches a GPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dsa_oracle.c")

MUTANTS = {
    "transposed_matrix": ("Srow[t[j - 1]]", "S[(size_t)t[j - 1] * A + q[i - 1]]"),
    "gap_costs_o_plus_ke": ("E = imax(E - e, H[j - 1] - o);", "E = imax(E - e, H[j - 1] - o - e);"),
    "tie_break_i_first": ("(j < *bj || (j == *bj && i < *bi))", "(i < *bi || (i == *bi && j < *bj))"),
    "global_row0_linear": ("return -(o + (int32_t)(j - 1) * e);", "return -((int32_t)(j) * e);"),
    "semiglobal_skips_col0_of_row_m": ("for (int64_t j = 0; j <= n; ++j) offer(H[j], m, j",
                                       "for (int64_t j = 1; j <= n; ++j) offer(H[j], m, j"),
    "traceback_D_before_I": ("} else if (v == AT(Fm, i, j)) {\n        state = 1;\n      } else {\n        state = 2;",
                             "} else if (v == AT(Em, i, j)) {\n        state = 2;\n      } else {\n        state = 1;"),
    "traceback_extend_before_open": ("if (AT(Fm, i, j) == AT(H, i - 1, j) - o) state = 0;",
                                     "if (AT(Fm, i, j) != AT(Fm, i - 1, j) - e) state = 0;"),
    "local_floor_missing": ("if (mode == ORC_LOCAL && h < 0) h = 0;\n      diag", "diag"),
    "profile_row_stride_dropped": ("P ? P + (size_t)(i - 1) * A", "P ? P + (size_t)(i - 1)"),
    "pair_window_offset_dropped": ("ts += J->pair_toff[p]; n = J->pair_tlen[p];",
                                   "n = J->pair_tlen[p];"),
    "pair_window_offset_absolute": ("ts += J->pair_toff[p]; n = J->pair_tlen[p];",
                                    "ts = J->t_codes + J->pair_toff[p]; n = J->pair_tlen[p];"),
    "pair_query_slice_shifted": ("const uint8_t* qs = J->q_codes + J->q_off[qi];",
                                 "const uint8_t* qs = J->q_codes + J->q_off[qi] + (qi > 0);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    before, after = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(before) == 1, f"mutation anchor for {name} not unique"
    c_path = tmp_path / f"{name}.c"
    c_path.write_text(src.replace(before, after))
    so_path = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", str(c_path), "-o",
                    str(so_path)], check=True)
    env = dict(os.environ, DSA_ORACLE_LIB=str(so_path))
    tests = [os.path.join(ROOT, "tests", "test_oracle_bruteforce.py"),
             os.path.join(ROOT, "tests", "test_oracle_golden.py"),
             os.path.join(ROOT, "tests", "test_oracle_pssm.py"),
             os.path.join(ROOT, "tests", "test_oracle_batch.py")]
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + tests,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} passed every pin:\n{r.stdout[-2000:]}"
