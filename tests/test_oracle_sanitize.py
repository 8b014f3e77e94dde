"""The oracle's pins under AddressSanitizer and UndefinedBehaviorSanitizer.

The C oracle is rebuilt with -fsanitize=address,undefined (any UB report
aborts) and the oracle pin tests run against it in a child process that
preloads libasan (leak checking off: the Python interpreter itself keeps
allocations alive at exit).  The exact-enumeration chi-squared tests are left
out for time; everything else that exercises the oracle's geometry, energy,
dE, tables, sweeps, clusters, qSRO model, replica exchange and specific heat
runs instrumented.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["test_oracle_geometry.py", "test_oracle_energy.py", "test_oracle_tables.py", "test_oracle_philox.py",
         "test_oracle_init_schedule.py", "test_oracle_sampler.py", "test_oracle_clusters.py", "test_oracle_qsro.py",
         "test_oracle_exchange.py", "test_oracle_cv.py", "test_oracle_fluct.py"]
SLOW = "not chi2 and not enumeration_sees and not wrong_temperature and not covariance_equals"


def test_oracle_pins_under_asan_ubsan():
    gcc = shutil.which("gcc")
    if not gcc:
        pytest.skip("gcc not available")
    asan = subprocess.run([gcc, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    if not os.path.isabs(asan) or not os.path.exists(asan):
        pytest.skip("libasan not available")
    sys.path.insert(0, ROOT)
    from oracle import build as ob
    ob.build(sanitize=True)
    env = dict(os.environ, SMCX_ORACLE_SANITIZE="1", LD_PRELOAD=asan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu", "-k", SLOW] + [
        os.path.join(ROOT, "tests", f) for f in FILES]
    probe = subprocess.run([sys.executable, "-c", "import oracle as O; print(O.lib()._name)"], env=env, cwd=ROOT,
                           capture_output=True, text=True)
    assert probe.returncode == 0 and probe.stdout.strip().endswith("libsmcx_oracle_san.so"), probe.stderr[-2000:]
    r = subprocess.run(cmd, env=env, cwd=ROOT, capture_output=True, text=True)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, tail
