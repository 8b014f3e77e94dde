"""Parity cases on the SMCX_DEBUG build (bounds-checked box, staging,
write-back, pair-count and store accesses that record a status word rather
than trap): a child process loads libsmcx_debug.so and runs a set of the
existing GPU parity tests; tests/conftest.py then requires a clean debug
status after each of them, and each must still match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_cases_on_debug_build():
    from paper_2503_12591_gb300 import build as lib_build
    lib_build.build(debug=True)
    env = dict(os.environ, SMCX_DEBUG="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
           os.path.join(ROOT, "tests", "test_gpu_parity.py"), os.path.join(ROOT, "tests", "test_gpu_anneal.py"),
           "-k", "not fullsize"]
    r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
