"""Oracle Philox4x32-10 pinned to an independent implementation.

The paper draws its trial random numbers with cuRAND (Method "Implementation
of SMC-GPU", random-number item) without naming the generator; this library
uses Philox4x32-10 (Salmon et al., SC'11).  The oracle's generator is checked
against ATen's ``philox_engine`` (shipped as a header with PyTorch), compiled
and run here on the same counters and keys.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O

ATEN_PROG = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
#include <cstdint>
int main() {
  unsigned long long seed, sub, off;
  while (std::scanf("%llu %llu %llu", &seed, &sub, &off) == 3) {
    at::Philox4_32 e(seed, sub, off);
    unsigned a = e(), b = e(), c = e(), d = e();
    std::printf("%u %u %u %u\n", a, b, c, d);
  }
  return 0;
}
"""


def _torch_include():
    try:
        import torch
    except Exception:
        return None
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    return inc if os.path.exists(os.path.join(inc, "ATen/core/PhiloxRNGEngine.h")) else None


@pytest.fixture(scope="module")
def aten_philox():
    inc = _torch_include()
    gxx = shutil.which("g++")
    if inc is None or gxx is None:
        pytest.skip("ATen headers or g++ unavailable")
    d = tempfile.mkdtemp()
    src = os.path.join(d, "p.cpp")
    exe = os.path.join(d, "p")
    with open(src, "w") as f:
        f.write(ATEN_PROG)
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", inc, src, "-o", exe], check=True)

    def run(triples):
        inp = "".join(f"{a} {b} {c}\n" for a, b, c in triples)
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return np.array([[int(x) for x in line.split()] for line in out.strip().splitlines()],
                        dtype=np.uint64)

    return run


def test_philox_matches_aten(aten_philox):
    rng = np.random.default_rng(12345)
    triples = []
    for i in range(400):
        seed = int(rng.integers(0, 2 ** 63)) * (1 + (i & 1))
        sub = int(rng.integers(0, 2 ** 63))
        off = int(rng.integers(0, 2 ** 63))
        if i < 4:  # edge counters
            seed, sub, off = [(0, 0, 0), (2 ** 64 - 1, 2 ** 64 - 1, 2 ** 64 - 1),
                              (1, 0, 0), (0, 1, 2 ** 32)][i]
        triples.append((seed % 2 ** 64, sub % 2 ** 64, off % 2 ** 64))
    ref = aten_philox(triples)
    for (seed, sub, off), want in zip(triples, ref):
        # ATen: key = seed (lo, hi); counter = (offset lo, offset hi, subseq lo, subseq hi)
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = O.philox(ctr, key)
        assert got.astype(np.uint64).tolist() == want.tolist()


def test_attempt_words_layout():
    seed, sweep = 0x1122334455667788, 0x0000000300000007
    for site in [0, 1, 2, 3, 12345, 2 ** 33 + 5]:
        j = site >> 1
        out = O.philox([j & 0xFFFFFFFF, (j >> 32) | (3 << 16), sweep & 0xFFFFFFFF, sweep >> 32],
                       [seed & 0xFFFFFFFF, seed >> 32])
        rd, ru = O.attempt_words(seed, sweep, 3, site)
        want = (out[2], out[3]) if site & 1 else (out[0], out[1])
        assert (rd, ru) == (int(want[0]), int(want[1]))


def test_direction_draw_uniform():
    # dir = floor(rd * z1 / 2^32) over many sites: chi-square against uniform
    z1 = 8
    counts = np.zeros(z1, np.int64)
    for s in range(20000):
        rd, _ = O.attempt_words(7, 11, 0, s)
        counts[(rd * z1) >> 32] += 1
    exp = counts.sum() / z1
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 30.0  # 7 dof, p ~ 1e-4
