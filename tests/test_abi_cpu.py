"""C ABI checks that need no GPU: the library loads, exports every function
include/smcx.h declares, and its host-side acceptance tables equal the
oracle's bit for bit (both follow the Metropolis acceptance equation of the
Supplementary, "Monte Carlo Simulation Algorithms")."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2503_12591_gb300 import build as lib_build
from paper_2503_12591_gb300 import smcx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return smcx.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(smcx_[a-z0-9_]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 15
    raw = ctypes.CDLL(smcx.LIB_PATH)
    for name in declared:
        assert hasattr(raw, name), f"{name} declared but not exported"
    assert declared <= set(smcx.exported_symbols()) | set(), "binding misses a declared entry point"


def test_version_and_error_message(lib):
    assert lib.smcx_version() >= 10000
    A = np.zeros(4, np.uint32)
    rc = lib.smcx_threshold_tables(-1.0, A.ctypes.data_as(ctypes.c_void_p), None, None)
    assert rc == smcx.E_INVALID_ARG
    assert lib.smcx_last_error()


@pytest.mark.parametrize("T", [1e-3, 250.0, 300.0, 800.0, 1000.0, 1200.0, 1500.0, 2500.0, 3000.0, 1e9])
def test_threshold_tables_equal_oracle(lib, T):
    A, nA, B = smcx.threshold_tables(T)
    oA, onA, oB = O.threshold_tables(T)
    assert nA == onA
    assert (A == oA).all() and (B == oB).all()
