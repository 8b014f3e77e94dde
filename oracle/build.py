"""Build the oracle shared library (plain C, gcc).

TEST INFRASTRUCTURE ONLY: the oracle is the serial CPU reference that the
tests, the smoke check and the benchmark's CPU-baseline leg compare against.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsmcx_oracle.so")
SRC = [os.path.join(HERE, "smcx_oracle.c")]
HDR = [os.path.join(HERE, "smcx_oracle.h")]


def build(force: bool = False) -> str:
    """Compile the oracle if it is missing or older than its sources."""
    os.makedirs(OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in SRC + HDR)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp]
    # OpenMP only splits the sites of one phase across threads (identical
    # results); without it the parallel entry point runs serially.
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + SRC + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + SRC + ["-lm"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
