"""Oracle Philox4x32-10 pinned to cuRAND's device generator.

The paper draws its trial random numbers with cuRAND (Method "Implementation
of SMC-GPU", random-number item).  cuRAND's Philox4_32_10 state started with
curand_init(seed, subsequence, offset) holds key = seed (lo, hi) and counter
= (offset / 4 lo, offset / 4 hi, subsequence lo, subsequence hi); for an
offset that is a multiple of 4, the first curand4() is the Philox block of
that counter.  A small program built here runs it on the GPU for random keys
and counters, and the oracle's generator must give the same four words.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

CURAND_PROG = r"""
#include <curand_kernel.h>
#include <cstdio>
#include <vector>
__global__ void blocks(const unsigned long long* in, uint4* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(in[3 * i], in[3 * i + 1], in[3 * i + 2], &st);
  out[i] = curand4(&st);
}
int main() {
  std::vector<unsigned long long> h;
  unsigned long long a, b, c;
  while (std::scanf("%llu %llu %llu", &a, &b, &c) == 3) {
    h.push_back(a);
    h.push_back(b);
    h.push_back(c);
  }
  const int n = (int)(h.size() / 3);
  if (n == 0) return 1;
  unsigned long long* d_in = nullptr;
  uint4* d_out = nullptr;
  if (cudaMalloc(&d_in, h.size() * sizeof(unsigned long long)) != cudaSuccess) return 2;
  if (cudaMalloc(&d_out, n * sizeof(uint4)) != cudaSuccess) return 2;
  cudaMemcpy(d_in, h.data(), h.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice);
  blocks<<<(n + 127) / 128, 128>>>(d_in, d_out, n);
  std::vector<uint4> o(n);
  if (cudaMemcpy(o.data(), d_out, n * sizeof(uint4), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  for (int i = 0; i < n; i++) std::printf("%u %u %u %u\n", o[i].x, o[i].y, o[i].z, o[i].w);
  cudaFree(d_in);
  cudaFree(d_out);
  return 0;
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_oracle_philox_matches_curand_device():
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc unavailable")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "c.cu"), os.path.join(d, "c")
    with open(src, "w") as f:
        f.write(CURAND_PROG)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", src, "-o", exe], check=True)
    rng = np.random.default_rng(2024)
    cases = []
    for i in range(300):
        key = [int(x) for x in rng.integers(0, 2 ** 32, 2)]
        ctr = [int(x) for x in rng.integers(0, 2 ** 32, 4)]
        ctr[1] &= (1 << 30) - 1  # offset = 4 (ctr0 + ctr1 2^32) stays below 2^64
        if i < 3:  # edge counters and keys
            key, ctr = [([0, 0], [0, 0, 0, 0]), ([2 ** 32 - 1] * 2, [2 ** 32 - 1, 2 ** 30 - 1, 2 ** 32 - 1, 2 ** 32 - 1]),
                        ([1, 0], [0, 0, 1, 0])][i]
        cases.append((key, ctr))
    inp = "".join(f"{k[0] | (k[1] << 32)} {c[2] | (c[3] << 32)} {4 * (c[0] | (c[1] << 32))}\n" for k, c in cases)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    got = [[int(x) for x in line.split()] for line in out.strip().splitlines()]
    assert len(got) == len(cases)
    for (key, ctr), want in zip(cases, got):
        assert O.philox(ctr, key).astype(np.uint64).tolist() == want
