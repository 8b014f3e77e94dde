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
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall", "-Wextra",
           "-o", tmp] + SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
