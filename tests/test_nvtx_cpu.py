"""NVTX ranges around the sweep-type entry points (a profiler-visible trace
of where each call enqueues its GPU work).

Runs without a GPU: a small NVTX injection library (tests/native/
nvtx_recorder.c) records every range push and pop, and the entry points are
called with a NULL handle, so each one opens its range, fails its argument
check with SMCX_E_INVALID_ARG and closes the range again.
"""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CALLS = ["smcx_sweep", "smcx_sweep_energies", "smcx_sweep_cv", "smcx_sweep_partial", "smcx_autotune",
         "smcx_energy", "smcx_batch_sweep", "smcx_batch_exchange", "smcx_batch_autotune",
         "smcx_batch_fluct_accumulate"]


def test_entry_points_open_and_close_their_ranges(tmp_path):
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    inc = "/usr/local/cuda/include"
    shim = tmp_path / "libnvtx_recorder.so"
    subprocess.run([gcc, "-O1", "-fPIC", "-shared", "-I", inc, "-o", str(shim),
                    os.path.join(ROOT, "tests", "native", "nvtx_recorder.c")], check=True)
    log = tmp_path / "nvtx.log"
    code = textwrap.dedent(f"""
        import ctypes as C, sys
        sys.path.insert(0, {ROOT!r})
        from paper_2503_12591_gb300 import smcx
        L = smcx.lib()
        v, d = C.c_void_p, C.c_double
        rc = [L.smcx_sweep(None, d(1000.0), 1, 1),
              L.smcx_sweep_energies(None, d(1000.0), 1, 1, None),
              L.smcx_sweep_cv(None, d(1000.0), 1, 1, None, None),
              L.smcx_sweep_partial(None, d(1000.0), 1, 1),
              L.smcx_autotune(None, d(1000.0), 1, None, None),
              L.smcx_energy(None, None),
              L.smcx_batch_sweep(None, None, 1, 1),
              L.smcx_batch_exchange(None, None, None, 1, 1, 1, None, None),
              L.smcx_batch_autotune(None, None, 1, None),
              L.smcx_batch_fluct_accumulate(None, 0, None)]
        assert all(r == smcx.E_INVALID_ARG for r in rc), rc
    """)
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(shim), SMCX_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT)
    lines = log.read_text().split("\n")[:-1]
    want = []
    for name in CALLS:
        want += [f"push {name}", "pop"]
    assert lines == want
