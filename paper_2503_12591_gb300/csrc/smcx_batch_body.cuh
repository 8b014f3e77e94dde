// Persistent batched sweep body: every replica, every sweep, every tile
// colour in one cooperative launch (temperature parallelism, Supplementary
// "Parallelization opportunities").  Included by smcx_batch.cu (per-trial
// directions) and smcx_sweep_bcc_dir.cu (shared-direction proposals, whose
// trial body and constant-memory offset table live in that translation unit).
#pragma once

#include "smcx_bcc_tile.cuh"

namespace smcx {
namespace bccfast {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a time limit; returns false if the grid must stop.
// Arrival: a CTA barrier, then one thread fences the CTA's writes and adds
// to the counter.  Departure: that thread sees the count, fences, and a CTA
// barrier releases the rest, so loads after it see every CTA's writes.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned target, int* status, long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    int ok = 1;
    const unsigned long long t0 = global_ns();
    while (true) {
      const unsigned v = *((volatile unsigned*)bar);
      if (v >= target) break;
      if (*((volatile int*)status) != 0) {
        ok = 0;
        break;
      }
      if ((long long)(global_ns() - t0) > timeout_ns) {
        atomicCAS(status, 0, SMCX_E_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// In each colour the CTAs take the pooled (replica, tile) items of that
// colour, CTA b the items b, b + G, b + 2G, ... (largest tiles first), then
// meet at the grid barrier.
template <int K, int NW, int PL, int SLOTS, int PROP>
__device__ __forceinline__ void batch_body(const Planes& Q, const LatDesc* __restrict__ descs,
                                           const int2* __restrict__ items, int n_items, int n_sweeps, unsigned* bar,
                                           int* status, long long timeout_ns, int skip_cta, int max_nA) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];
  uint8_t* box = smem;
  uint32_t* sA = reinterpret_cast<uint32_t*>(smem + 2 * SUB);
  uint32_t* sB = sA + max_nA;
  unsigned epoch = 0;
  for (int s = 0; s < n_sweeps; s++)
    for (int tc = 0; tc < 8; tc++) {
      for (int e = blockIdx.x; e < n_items; e += gridDim.x) {
        const int2 it = items[e];
        const LatDesc D = descs[it.x];
        bcc_tile_pass<K, NW, PL, SLOTS, PROP>(D, Q, tc, it.y, D.sweep + (unsigned long long)s, box, sA, sB,
                                              s_stat);
      }
      if ((int)blockIdx.x == skip_cta) return;
      epoch++;
      if (!grid_barrier(bar, epoch * gridDim.x, status, timeout_ns)) return;
    }
}

// 128-thread CTAs (one or two link-cell slots per thread), and 256-thread
// CTAs for tiles of up to 256 slots (6^3 with link cells of 3): one slot per
// thread, so a tile's phases take half the sequential steps of two slots.
template <int K, int NW, int PL, int SLOTS, int PROP>
__global__ void __launch_bounds__(128, 6)
    k_bcc_batch(const Planes Q, const LatDesc* __restrict__ descs, const int2* __restrict__ items, int n_items,
                int n_sweeps, unsigned* bar, int* status, long long timeout_ns, int skip_cta, int max_nA) {
  batch_body<K, NW, PL, SLOTS, PROP>(Q, descs, items, n_items, n_sweeps, bar, status, timeout_ns, skip_cta, max_nA);
}
template <int K, int NW, int PL, int PROP>
__global__ void __launch_bounds__(256, 3)
    k_bcc_batch256(const Planes Q, const LatDesc* __restrict__ descs, const int2* __restrict__ items, int n_items,
                   int n_sweeps, unsigned* bar, int* status, long long timeout_ns, int skip_cta, int max_nA) {
  batch_body<K, NW, PL, 1, PROP>(Q, descs, items, n_items, n_sweeps, bar, status, timeout_ns, skip_cta, max_nA);
}

using BatchKernelFn = void (*)(const Planes, const LatDesc*, const int2*, int, int, unsigned*, int*, long long, int,
                               int);

}  // namespace bccfast

// The shared-direction batch kernel (4 shells, M <= 4, two byte planes, one
// link-cell slot per thread) for 128- or 256-thread CTAs.
bccfast::BatchKernelFn batch_dir_kernel(int threads);  // smcx_sweep_bcc_dir.cu

}  // namespace smcx
