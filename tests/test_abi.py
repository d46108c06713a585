"""The C-ABI library builds, loads and exports every entry point include/dsa.h declares.

No compute runs here (no GPU needed): creating a context on a machine without
a GPU must return an error code, not crash."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1701_01575_gb300 import build, dsa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dsa.h")


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(dsa_[a-z_0-9]+)\s*\(",
                                 text, flags=re.M)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("dsa_db_load", "dsa_align_batch", "dsa_traceback", "dsa_align", "dsa_res_get"):
        assert name in syms
    assert set(syms) == set(dsa.SYMBOLS)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # dsa_hit: 8 x 32-bit, 2 x 64-bit, 2 x 32-bit; dsa_pair: 2 x 32, 64, 2 x 32
    assert dsa.HIT_DTYPE.itemsize == 56 and dsa.HIT_DTYPE.fields["t_offset"][1] == 32
    assert dsa.PAIR_DTYPE.itemsize == 24 and dsa.PAIR_DTYPE.fields["t_offset"][1] == 8
    from paper_1701_01575_gb300 import workloads as W
    assert W.PAIR_DTYPE.itemsize == dsa.PAIR_DTYPE.itemsize


def test_no_gpu_gives_error_code_not_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    dsa.load_library(build.LIB)
    h = ctypes.c_void_p()
    rc = dsa._lib.dsa_create(ctypes.byref(h), 0, 0, None)
    assert rc in (dsa.ERR_CUDA, dsa.ERR_INVALID_ARG)
    assert dsa._lib.dsa_last_error()


def test_null_arguments_rejected(lib):
    dsa.load_library(build.LIB)
    assert dsa._lib.dsa_create(None, 0, 0, None) == dsa.ERR_INVALID_ARG
    assert dsa._lib.dsa_db_load(None, None, None, 0, 4, None) == dsa.ERR_INVALID_ARG
    assert dsa._lib.dsa_res_stats(None, None, None) == dsa.ERR_INVALID_ARG
