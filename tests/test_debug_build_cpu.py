"""The SMCX_DEBUG build of the CUDA library (in-kernel bounds checks that
record a status word instead of trapping) compiles for sm_103a and carries
its status entry point; the normal build refuses that entry point.  Runs on
the CPU: nvcc cross-compiles, and smcx_debug_status is checked only for the
paths that need no GPU.  tests/test_gpu_debug_build.py runs parity cases on
the debug build on a GPU."""
import ctypes as C
import os
import shutil

import pytest

from paper_2503_12591_gb300 import build as lib_build
from paper_2503_12591_gb300 import smcx


def test_debug_build_compiles_and_reports():
    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available")
    path = lib_build.build(debug=True)
    assert path.endswith("libsmcx_debug.so") and os.path.exists(path)
    dbg = C.CDLL(path)
    dbg.smcx_debug_status.restype = C.c_int
    dbg.smcx_debug_status.argtypes = [C.c_void_p]
    info = (C.c_uint64 * 2)()
    assert dbg.smcx_debug_status(None) == smcx.E_INVALID_ARG
    # the debug path synchronises the device first: no GPU here -> CUDA error,
    # with a GPU -> OK; never "unsupported"
    assert dbg.smcx_debug_status(info) != smcx.E_UNSUPPORTED
    normal = smcx.lib()
    assert normal.smcx_debug_status(info) == smcx.E_UNSUPPORTED
