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


LIB_SAN = os.path.join(OUT_DIR, "libsmcx_oracle_san.so")
SAN_FLAGS = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g"]


def build(force: bool = False, sanitize: bool = False) -> str:
    """Compile the oracle if it is missing or older than its sources.
    sanitize=True builds a separate copy with AddressSanitizer and
    UndefinedBehaviorSanitizer (loaded by processes that preload libasan)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = LIB_SAN if sanitize else LIB
    newest = max(os.path.getmtime(p) for p in SRC + HDR)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    opt = SAN_FLAGS + ["-O1"] if sanitize else ["-O2"]
    base = ["gcc"] + opt + ["-std=c99", "-fPIC", "-shared", "-Wall", "-Wextra", "-o", tmp]
    # OpenMP only splits the sites of one phase across threads (identical
    # results); without it the parallel entry point runs serially.
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + SRC + ["-lm"], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base + SRC + ["-lm"], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
