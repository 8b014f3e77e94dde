// Device-side building blocks shared by the kernel translation units.
#pragma once

#include <stdint.h>

#include "smcx_internal.h"

namespace smcx {

// ---- SMCX_DEBUG: in-kernel bounds checks --------------------------------
// Built with -DSMCX_DEBUG (the library's debug build, libsmcx_debug.so), the
// checked accesses below test their index against the buffer's extent; an
// index outside it skips the access (a load returns 0) and records a tag and
// the index in this translation unit's device status words, which
// smcx_debug_status reads and clears.  Nothing traps or returns early, so
// every barrier of the kernel is still reached.  In the normal build the
// helpers are the plain access.
enum DebugTag : unsigned {
  kDbgBccBox = 1,      // BCC tile pass: trial loads and stores in the box
  kDbgBccStage = 2,    // BCC tile pass: staging stores
  kDbgBccWrite = 3,    // BCC tile pass: write-back loads from the box
  kDbgBccDir = 4,      // BCC tile pass: phase-direction table
  kDbgTileBox = 5,     // generic tile sweep: box accesses
  kDbgFccBox = 6,      // FCC tile pass: box accesses
  kDbgPairHist = 7,    // pair counts: histogram bin
  kDbgSite = 8,        // global-memory kernels: site index
  kDbgQsroBox = 9,     // qSRO tile passes: box accesses
};
#ifdef SMCX_DEBUG
namespace dbg {
static __device__ unsigned long long g_status[2];  // tag of the first failure, its index
__device__ __forceinline__ bool in_bounds(long long i, long long n, unsigned tag) {
  if (i >= 0 && i < n) return true;
  if (atomicCAS(&g_status[0], 0ull, (unsigned long long)tag) == 0ull) g_status[1] = (unsigned long long)i;
  return false;
}
// Host reader of this translation unit's status words (registered below).
static int read_and_clear(unsigned long long* out) {
  const unsigned long long zero[2] = {0ull, 0ull};
  if (cudaMemcpyFromSymbol(out, g_status, sizeof(zero)) != cudaSuccess) return -1;
  if (cudaMemcpyToSymbol(g_status, zero, sizeof(zero)) != cudaSuccess) return -1;
  return 0;
}
int register_reader(int (*reader)(unsigned long long*));  // smcx_api.cu
static const int g_registered = register_reader(&read_and_clear);
}  // namespace dbg
#endif
template <class T, class I>
__device__ __forceinline__ T ld_chk(const T* p, I i, I n, unsigned tag) {
#ifdef SMCX_DEBUG
  if (!dbg::in_bounds((long long)i, (long long)n, tag)) return T(0);
#endif
  return p[i];
}
template <class T, class I>
__device__ __forceinline__ void st_chk(T* p, I i, I n, unsigned tag, T v) {
#ifdef SMCX_DEBUG
  if (!dbg::in_bounds((long long)i, (long long)n, tag)) return;
#endif
  p[i] = v;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies with a word permutation and key xor; the key is
// bumped by the Weyl constants between rounds.
__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = mulhi32(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = mulhi32(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Random words of the pair (site id >> 1) in sweep `sweep` of replica `rep`.
__device__ __forceinline__ uint4 attempt_block(unsigned long long gid, unsigned long long sweep,
                                               int rep, uint32_t seed_lo, uint32_t seed_hi) {
  const unsigned long long j = gid >> 1;
  return philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32) | ((uint32_t)rep << 16),
                                  (uint32_t)sweep, (uint32_t)(sweep >> 32)),
                       make_uint2(seed_lo, seed_hi));
}

// Shell-1 direction shared by every trial of one (sweep, tile, intra colour)
// under shared-direction proposals: Philox counter (tile, (ic >> 1) |
// replica << 16, sweep lo, sweep hi | 2^30), key = seed; word 0 (even ic) or
// word 2 (odd ic); floor(word * z1 / 2^32).
__device__ __forceinline__ uint4 phase_direction_block(uint32_t seed_lo, uint32_t seed_hi, unsigned long long sweep,
                                                       int rep, unsigned tile, int ic_pair) {
  return philox4x32_10(make_uint4(tile, (uint32_t)ic_pair | ((uint32_t)rep << 16), (uint32_t)sweep,
                                  (uint32_t)(sweep >> 32) | 0x40000000u),
                       make_uint2(seed_lo, seed_hi));
}
__device__ __forceinline__ int phase_direction(uint32_t seed_lo, uint32_t seed_hi, unsigned long long sweep, int rep,
                                               unsigned tile, int ic, int z1) {
  const uint4 r = phase_direction_block(seed_lo, seed_hi, sweep, rep, tile, ic >> 1);
  return (int)__umulhi((ic & 1) ? r.z : r.x, (uint32_t)z1);
}

// Block-shared proposals: the shell-1 direction of phase ic shared by the
// tiles of one block (a pair of consecutive tiles of colour tc, numbered in
// launch order (jz, jy, jx) within the colour): Philox counter (block | tc <<
// 28, (ic >> 1) | replica << 16, sweep lo, sweep hi | 2^29), key = seed;
// word 0 (even ic) or word 2 (odd ic); floor(word * z1 / 2^32).
__device__ __forceinline__ uint4 block_direction_block(uint32_t seed_lo, uint32_t seed_hi, unsigned long long sweep,
                                                       int rep, int tc, unsigned block, int ic_pair) {
  return philox4x32_10(make_uint4(block | ((uint32_t)tc << 28), (uint32_t)ic_pair | ((uint32_t)rep << 16),
                                  (uint32_t)sweep, (uint32_t)(sweep >> 32) | 0x20000000u),
                       make_uint2(seed_lo, seed_hi));
}
__device__ __forceinline__ int block_direction(uint32_t seed_lo, uint32_t seed_hi, unsigned long long sweep, int rep,
                                               int tc, unsigned block, int ic, int z1) {
  const uint4 r = block_direction_block(seed_lo, seed_hi, sweep, rep, tc, block, ic >> 1);
  return (int)__umulhi((ic & 1) ? r.z : r.x, (uint32_t)z1);
}

// Shell sizes of the cubic lattices (BCC 8, 6, 12, 24; FCC 12, 6, 24).
__host__ __device__ constexpr int shell_size(int kind, int k) {
  return kind == kBCC ? (k == 0 ? 8 : k == 1 ? 6 : k == 2 ? 12 : 24)
                      : (k == 0 ? 12 : k == 1 ? 6 : 24);
}
__host__ __device__ constexpr int vec_count(int kind, int K) {
  return K <= 0 ? 0 : vec_count(kind, K - 1) + shell_size(kind, K - 1);
}
__host__ __device__ constexpr int cell_sites(int kind) { return kind == kBCC ? 2 : 4; }

// Metropolis decision with the two-level integer table (see smcx.h).
__device__ __forceinline__ bool metropolis_accept(int dE, uint32_t u, const uint32_t* A, int nA,
                                                  const uint32_t* B) {
  if (dE <= 0) return true;
  const int hi = dE >> 10;
  if (hi >= nA) return false;
  const uint32_t thr =
      (uint32_t)(((unsigned long long)A[hi] * (unsigned long long)B[dE & (kNB - 1)]) >> 32);
  return u < thr;
}

// Add a thread's trial counts to the CTA's shared counters (accepted,
// same-species, sum of accepted dE): summed across the warp first, so that
// each warp makes one shared atomic per counter.  Every lane of the warp
// must call it.
__device__ __forceinline__ void add_stats_warp(unsigned long long* s_stat, unsigned acc, unsigned same,
                                               long long dsum) {
  acc = __reduce_add_sync(0xffffffffu, acc);
  same = __reduce_add_sync(0xffffffffu, same);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_stat[0], (unsigned long long)acc);
    atomicAdd(&s_stat[1], (unsigned long long)same);
    atomicAdd(&s_stat[2], (unsigned long long)dsum);
  }
}

__device__ __forceinline__ int wrap_add(int x, int d, int n) {
  int t = x + d;
  t += (t < 0) ? n : 0;
  t -= (t >= n) ? n : 0;
  return t;
}

// One species id of site `gid` from the lattice store.
__device__ __forceinline__ int load_site(const uint8_t* sites, long long gid, int storage) {
  if (storage == SMCX_INT8) return sites[gid];
  const uint8_t byte = sites[gid >> 1];
  return (gid & 1) ? (byte >> 4) : (byte & 15);
}

// Launch parameters of the sweep kernels (passed by value: they live in the
// kernel parameter bank, so concurrent launches never share them).
struct SweepParams {
  uint8_t* sites;
  const uint32_t* thr;         // A[kNA] then B[kNB]
  const int32_t* wtab;         // W[a][b][k][c] then X[a][b]
  unsigned long long* stats;   // trials, accepts, same-species, sum of accepted dE
  int n[3];
  int nt[3];
  int ntc[3];                  // tiles of this launch's colour on each axis
  int tc;                      // tile colour (bit a = parity on axis a)
  int L, h, ring;
  int BX, BY, BZ;              // shared-memory box extents (cells)
  int M, nA, storage, replica;
  uint32_t seed_lo, seed_hi;
  unsigned long long sweep;
  int ic;                      // link-cell kernel: intra colour of the launch
  int proposal;                // 0: direction per trial; 1: per (sweep, tile, intra colour)
  int off[4][kMaxVec];         // box offsets of neighbours, per centre sublattice
  int poff[4][kMaxZ1];         // box offset of the partner, per sublattice/direction
  int psub[4][kMaxZ1];         // partner sublattice
  signed char gd[4][kMaxVec][4];  // global (dx, dy, dz, b') of neighbours
  signed char gp[4][kMaxZ1][4];   // global (dx, dy, dz, b') of partners
};

// Generic tiled kernels: stage the cells [t0 - h, t0 + ts + h) of each axis
// (periodic; the halo never exceeds one lattice edge) into a box of int8
// species, cell (xs, ys, zs) at ((zs BY + ys) BX + xs) m.  One box column per
// lane, warp w the rows w U .. w U + U - 1, w U + nwarp U, ... of each plane;
// the loads of U rows are issued before any is unpacked.  blockDim is a
// multiple of 32; every thread of the CTA takes part.
template <int m>
__device__ __forceinline__ void stage_generic(const SweepParams& P, int8_t* box, const int* t0, const int* ts, int h) {
  constexpr int U = 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ex = ts[0] + 2 * h, ey = ts[1] + 2 * h, ez = ts[2] + 2 * h;
  for (int zs = 0; zs < ez; zs++) {
    const long long zrow = (long long)wrap_add(t0[2] - h, zs, P.n[2]) * P.n[1];
    for (int ys0 = warp * U; ys0 < ey; ys0 += nwarp * U)
      for (int xs0 = 0; xs0 < ex; xs0 += 32) {
        const int xs = xs0 + lane;
        const int gx = xs < ex ? wrap_add(t0[0] - h, xs, P.n[0]) : 0;
        uint32_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          v[u] = 0;
          if (ys < ey && xs < ex) {
            const long long cell = (zrow + wrap_add(t0[1] - h, ys, P.n[1])) * P.n[0] + gx;
            if (P.storage == SMCX_INT8)
              v[u] = m == 4 ? *reinterpret_cast<const uint32_t*>(P.sites + 4 * cell)
                            : (uint32_t)(*reinterpret_cast<const uint16_t*>(P.sites + 2 * cell));
            else
              v[u] = m == 4 ? (uint32_t)(*reinterpret_cast<const uint16_t*>(P.sites + 2 * cell))
                            : (uint32_t)P.sites[cell];
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          if (ys < ey && xs < ex) {
            const int bi = ((zs * P.BY + ys) * P.BX + xs) * m;
#pragma unroll
            for (int b = 0; b < m; b++)
              box[bi + b] = (int8_t)(P.storage == SMCX_INT8 ? (v[u] >> (8 * b)) & 0xFFu : (v[u] >> (4 * b)) & 15u);
          }
        }
      }
  }
}

// Generic tiled kernels: write the tile and its partner ring (rg cells) back
// from the box staged by stage_generic with halo h.  One column per lane,
// warp w the rows w, w + nwarp, ... of each plane.
template <int m>
__device__ __forceinline__ void write_back_generic(const SweepParams& P, const int8_t* box, const int* t0,
                                                   const int* ts, int h, int rg) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int wx = ts[0] + 2 * rg, wy = ts[1] + 2 * rg, wz = ts[2] + 2 * rg;
  for (int zw = 0; zw < wz; zw++) {
    const long long zrow = (long long)wrap_add(t0[2] - rg, zw, P.n[2]) * P.n[1];
    const int zs = zw + h - rg;
    for (int yw = warp; yw < wy; yw += nwarp) {
      const long long rbase = (zrow + wrap_add(t0[1] - rg, yw, P.n[1])) * P.n[0];
      const int ys = yw + h - rg;
      for (int xw = lane; xw < wx; xw += 32) {
        const long long cell = rbase + wrap_add(t0[0] - rg, xw, P.n[0]);
        const int bi = ((zs * P.BY + ys) * P.BX + (xw + h - rg)) * m;
        if (P.storage == SMCX_INT8) {
#pragma unroll
          for (int b = 0; b < m; b++) P.sites[cell * m + b] = (uint8_t)box[bi + b];
        } else {
#pragma unroll
          for (int q = 0; q < m / 2; q++)
            P.sites[cell * (m / 2) + q] = (uint8_t)(box[bi + 2 * q] | (box[bi + 2 * q + 1] << 4));
        }
      }
    }
  }
}

}  // namespace smcx
