// BCC tile pass specialised for throughput (M <= 8 species, K <= 4 shells,
// tiles up to 20 cells so that tile + 2-cell halo fits a 24^3 box).  Used by
// the single-lattice sweep (smcx_sweep_bcc.cu) and the batched persistent
// sweep (smcx_batch.cu).
//
// Same trials, same order of phases, same Philox words and the same integer
// arithmetic as k_tile_sweep in smcx_sweep.cu: the result is bit-identical;
// only the data layout and the instruction mix differ.
//
//  * Shared memory holds one byte per site, the species id times 8, in two
//    sublattice arrays with padded pitches (25-byte rows, 613-byte planes)
//    and a lane order that put the 32 centre sites of a warp on 32 banks.
//    The box pitches are compile-time constants, so every neighbour load is a
//    single LDS with an immediate offset from the centre (or partner)
//    address.
//  * Each neighbour adds 1 << (8 sigma) to a per-shell register of byte
//    counters (biased by 0x80 per byte): the s environment adds, the s'
//    environment subtracts, so byte c ends as 0x80 + n_k(s)[c] - n_k(s')[c].
//  * dE = G_b - G_a with G_p = sum_k sum_c V_k[p][c] D_k[c]: dp4a against the
//    byte planes of V held in the kernel parameter bank (uniform operands).
//  * A thread owns SLOTS link-cell slots of the tile for the whole pass; the
//    Philox block of a cell (two sites) is drawn once in the b = 0 phase and
//    its second half used in the b = 1 phase that immediately follows.
#pragma once

#include "smcx_device.cuh"

namespace smcx {

namespace bccfast {

constexpr int PX = 25;             // row pitch (cells)
constexpr int PP = 613;            // plane pitch (bytes: 24 rows + 13 bytes of padding)
constexpr int PZ = 24;             // planes
constexpr int SUB = PP * PZ;       // bytes per sublattice array
constexpr int BOX = 24;            // usable box edge (tile <= 20 with halo 2)

// Lane order of the 5^3 link-cell slots of a 20-cell tile (L = 4) on a
// 128-thread CTA: slot kSlotOrder[t] for thread t (255: none).  Slot q =
// (qx, qy, qz) = (q % 5, q / 5 % 5, q / 25) starts at byte qx 4 + qy 4 PX +
// qz 4 PP of the box, i.e. word qx + qy PX + qz PP; the order gives the 32
// lanes of every warp 32 different banks, so a neighbour load at a common
// offset (all loads of the centre environment) is one wavefront.  Any order
// gives the same result: the trials of a phase are independent.
#define SMCX_BCC_SLOT_ORDER                                                                                          \
  0, 1, 2, 3, 4, 21, 22, 23, 24, 29, 46, 15, 16, 17, 18, 19, 40, 41, 10, 11, 12, 13, 14, 35, 36, 5, 6, 7, 8, 9, 30, 31, 32, 33, 34, 55, 20, 25, 26, 27, 28, 45, 50, 47, 48, 49, 54, 71, 72, 73, 42, 43, 44, 65, 66, 67, 68, 37, 38, 39, 60, 61, 62, 63, 64, 85, 86, 87, 56, 57, 58, 59, 80, 81, 82, 51, 52, 53, 70, 75, 76, 77, 74, 79, 96, 97, 98, 99, 104, 69, 90, 91, 92, 93, 94, 115, 116, 117, 118, 119, 88, 89, 110, 111, 112, 113, 114, 83, 84, 105, 106, 107, 108, 109, 78, 95, 100, 101, 102, 103, 120, 121, 122, 123, 124, 255, 255, 255
constexpr unsigned char kSlotOrder[128] = {SMCX_BCC_SLOT_ORDER};
static __constant__ unsigned char c_slot_order[128] = {SMCX_BCC_SLOT_ORDER};
__host__ __device__ constexpr bool slot_order_ok() {
  for (int w = 0; w < 4; w++) {
    bool seen[32] = {};
    for (int l = 0; l < 32; l++) {
      const int q = kSlotOrder[32 * w + l];
      if (q == 255) continue;
      const int bank = (q % 5 + PX * (q / 5 % 5) + PP * (q / 25)) % 32;
      if (seen[bank]) return false;
      seen[bank] = true;
    }
  }
  bool used[125] = {};
  for (int t = 0; t < 128; t++) {
    const int q = kSlotOrder[t];
    if (q == 255) continue;
    if (q >= 125 || used[q]) return false;
    used[q] = true;
  }
  for (int q = 0; q < 125; q++)
    if (!used[q]) return false;
  return true;
}
static_assert(slot_order_ok(), "slot order must cover the 125 slots with distinct banks per warp");
constexpr int MAXPLANES = 3;

// Byte planes of the EPI table, shared by every lattice of a launch:
// P[j][k][p][w] holds bytes j of V_k[p][4w .. 4w+3] (planes below the top one
// unsigned, the top plane signed).
struct Planes {
  uint32_t P[MAXPLANES][kMaxShells][kMaxSweepM][2];
  // Rows of V differences for shared-direction trials (M <= 4, 4 shells):
  // R[a * 4 + b][k] holds the low bytes (unsigned), R[a * 4 + b][4 + k] the
  // high bytes (signed) of T_k[c] = V_k[b][c] - V_k[a][c], c = 0..3; valid
  // (rows = 1) when every |T| < 2^15.
  uint32_t R[16][8];
  int rows;
};

// One lattice as the tile pass sees it.
struct LatDesc {
  uint8_t* sites;
  const uint32_t* thr;          // A[kNA] then B[kNB] at this lattice's temperature
  unsigned long long* stats;    // trials, accepts, same-species, sum dE
  int n[3], nt[3];
  int L, NQ;                    // link-cell edge; link-cell slots per tile axis
  int nA, storage, replica;
  uint32_t seed_lo, seed_hi;
  unsigned long long sweep;     // cumulative index of the first sweep of the call
  int M;                        // species count (pair counting)
  int proposal;                 // 0: direction per trial; 1: per (sweep, tile, intra colour); 2: per block
};

// 50 BCC neighbour vectors (half units) of shells 1..4 with their shell.
struct Vec {
  int x, y, z, k;
};
__host__ __device__ constexpr int bcc_shell_of(int x, int y, int z) {
  return (x * x + y * y + z * z) == 3 ? 0 : (x * x + y * y + z * z) == 4 ? 1 : (x * x + y * y + z * z) == 8 ? 2
         : (x * x + y * y + z * z) == 11 ? 3 : -1;
}
struct VecTable {
  Vec v[50];
  int n;
};
__host__ __device__ constexpr VecTable make_vecs() {
  VecTable t{};
  t.n = 0;
  for (int x = -3; x <= 3; x++)
    for (int y = -3; y <= 3; y++)
      for (int z = -3; z <= 3; z++) {
        const bool odd = (x & 1) && (y & 1) && (z & 1);
        const bool even = !(x & 1) && !(y & 1) && !(z & 1);
        if (!(odd || even)) continue;
        const int k = bcc_shell_of(x, y, z);
        if (k < 0) continue;
        t.v[t.n] = Vec{x, y, z, k};
        t.n++;
      }
  return t;
}
__host__ __device__ constexpr int floor2(int p) { return p >= 0 ? p / 2 : -((1 - p) / 2); }
// byte offset (in the box) from a site of sublattice B to its neighbour along v
__host__ __device__ constexpr int nb_offset(int B, int x, int y, int z) {
  return (((B + x) & 1) - B) * SUB + floor2(B + z) * PP + floor2(B + y) * PX + floor2(B + x);
}

__device__ __forceinline__ int dp4a_su(int a, uint32_t b, int c) {
  int d;
  asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp4a_ss(int a, uint32_t b, int c) {
  int d;
  asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Accumulate the environment of a site of sublattice B at box index `c`
// into the per-shell byte counters (SIGN = +1 for s, -1 for s').
template <int B, int K, int NW, int SIGN>
__device__ __forceinline__ void gather(const uint8_t* box, int c, uint32_t (&h)[kMaxShells][2]) {
  constexpr VecTable T = make_vecs();
#pragma unroll
  for (int j = 0; j < T.n; j++) {
    const int k = T.v[j].k;
    if (k >= K) continue;
    const uint32_t v = ld_chk(box, c + nb_offset(B, T.v[j].x, T.v[j].y, T.v[j].z), 2 * SUB, kDbgBccBox);
    if (NW == 1) {
      const uint32_t one = 1u << v;
      if (SIGN > 0) h[k][0] += one; else h[k][0] -= one;
    } else {
      uint32_t lo, hi;
      asm("shl.b32 %0, 1, %1;" : "=r"(lo) : "r"(v));
      asm("shl.b32 %0, 1, %1;" : "=r"(hi) : "r"(v - 32u));
      if (SIGN > 0) {
        h[k][0] += lo;
        h[k][1] += hi;
      } else {
        h[k][0] -= lo;
        h[k][1] -= hi;
      }
    }
  }
}

template <int NW>
__device__ __forceinline__ void add_one(uint32_t (&h)[2], uint32_t v, int sign) {
  uint32_t lo, hi;
  asm("shl.b32 %0, 1, %1;" : "=r"(lo) : "r"(v));
  if (NW == 1) {
    h[0] += sign > 0 ? lo : (uint32_t)(-(int)lo);
  } else {
    asm("shl.b32 %0, 1, %1;" : "=r"(hi) : "r"(v - 32u));
    h[0] += sign > 0 ? lo : (uint32_t)(-(int)lo);
    h[1] += sign > 0 ? hi : (uint32_t)(-(int)hi);
  }
}

// One trial at box index s (sublattice B) with Philox words (rd, ru).
template <int B, int K, int NW, int PL>
__device__ __forceinline__ void trial(uint8_t* box, int s, uint32_t rd, uint32_t ru, const Planes& P, int nA,
                                      const uint32_t* sA, const uint32_t* sB, unsigned& acc, unsigned& same,
                                      long long& dsum) {
  const int dir = (int)(rd >> 29);  // floor(rd * 8 / 2^32)
  // shell-1 vector (+-1,+-1,+-1): bit 2 -> x, bit 1 -> y, bit 0 -> z
  const int dx = ((dir >> 2) & 1) - 1 + B, dy = ((dir >> 1) & 1) - 1 + B, dz = (dir & 1) - 1 + B;
  const int sp = s + (1 - 2 * B) * SUB + dz * PP + dy * PX + dx;
  const uint32_t a8 = ld_chk(box, s, 2 * SUB, kDbgBccBox), b8 = ld_chk(box, sp, 2 * SUB, kDbgBccBox);
  if (a8 == b8) {
    same++;
    return;
  }
  uint32_t h[kMaxShells][2];
#pragma unroll
  for (int k = 0; k < kMaxShells; k++) {
    h[k][0] = 0x80808080u;
    h[k][1] = 0x80808080u;
  }
  gather<B, K, NW, +1>(box, s, h);
  gather<1 - B, K, NW, -1>(box, sp, h);
  // the s-s' bond is not part of either environment after the swap
  add_one<NW>(h[0], b8, -1);
  add_one<NW>(h[0], a8, +1);
  // G_p = sum_k sum_c V_k[p][c] D_k[c]
  const int a = (int)(a8 >> 3), b = (int)(b8 >> 3);
  int Ga = 0, Gb = 0;
#pragma unroll
  for (int p = 0; p < 4 * NW; p++) {
    int acc0 = 0, acc1 = 0, acc2 = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
      for (int w = 0; w < NW; w++) {
        const int d = (int)(h[k][w] ^ 0x80808080u);
        if (PL == 1) {
          acc0 = dp4a_ss(d, P.P[0][k][p][w], acc0);
        } else {
          acc0 = dp4a_su(d, P.P[0][k][p][w], acc0);
          if (PL == 2) {
            acc1 = dp4a_ss(d, P.P[1][k][p][w], acc1);
          } else {
            acc1 = dp4a_su(d, P.P[1][k][p][w], acc1);
            acc2 = dp4a_ss(d, P.P[2][k][p][w], acc2);
          }
        }
      }
    }
    const int G = acc0 + (acc1 << 8) + (acc2 << 16);
    Ga = (p == a) ? G : Ga;
    Gb = (p == b) ? G : Gb;
  }
  const int dE = Gb - Ga;
  if (metropolis_accept(dE, ru, sA, nA, sB)) {
    st_chk(box, s, 2 * SUB, kDbgBccBox, (uint8_t)b8);
    st_chk(box, sp, 2 * SUB, kDbgBccBox, (uint8_t)a8);
    acc++;
    dsum += dE;
  }
}

// ---- shared-direction proposals ------------------------------------------
// With one direction per (sweep, tile, intra colour) every lane of a phase
// has its partner at the same offset, so the union of the two environments
// (68 distinct sites for 4 BCC shells, instead of 2 x 50 loads) is the same
// for the whole warp: each site adds to the counter of its shell around s and
// subtracts from the counter of its shell around s'.  The 8 directions are
// reflections of direction 7 = (+,+,+), which preserve both shells, so one
// entry list per sublattice (shells fixed at compile time) serves all of
// them; only the box offsets depend on the direction, and are read from a
// constant-memory table at a warp-uniform index.
struct UEntry {
  int x, y, z, k1, k2;  // half-unit vector from s; shell around s / s' (-1: none)
};
struct UTable {
  UEntry e[96];
  int n;
};
__host__ __device__ constexpr int bcc_shell_k(int x, int y, int z, int K) {
  const bool odd = (x & 1) && (y & 1) && (z & 1);
  const bool even = !(x & 1) && !(y & 1) && !(z & 1);
  if (!(odd || even)) return -1;
  const int k = bcc_shell_of(x, y, z);
  return k < K ? k : -1;
}
// union of the environments of s and s' = s + (1,1,1) (direction 7)
template <int K>
__host__ __device__ constexpr UTable make_union7() {
  UTable t{};
  t.n = 0;
  for (int x = -4; x <= 4; x++)
    for (int y = -4; y <= 4; y++)
      for (int z = -4; z <= 4; z++) {
        if ((x == 0 && y == 0 && z == 0) || (x == 1 && y == 1 && z == 1)) continue;
        const int k1 = bcc_shell_k(x, y, z, K);
        const int k2 = bcc_shell_k(x - 1, y - 1, z - 1, K);
        if (k1 < 0 && k2 < 0) continue;
        t.e[t.n] = UEntry{x, y, z, k1, k2};
        t.n++;
      }
  return t;
}
constexpr int kUnionMax = 72;
struct UnionOffsets {
  int off[2][8][kUnionMax];  // box offset of entry j reflected into direction d
  int poff[2][8];            // partner offset
};
__host__ __device__ constexpr UnionOffsets make_union_offsets() {
  UnionOffsets u{};
  constexpr UTable T = make_union7<4>();
  for (int B = 0; B < 2; B++)
    for (int d = 0; d < 8; d++) {
      const int sx = (d >> 2) & 1 ? 1 : -1, sy = (d >> 1) & 1 ? 1 : -1, sz = d & 1 ? 1 : -1;
      u.poff[B][d] = nb_offset(B, sx, sy, sz);
      for (int j = 0; j < T.n; j++) u.off[B][d][j] = nb_offset(B, sx * T.e[j].x, sy * T.e[j].y, sz * T.e[j].z);
    }
  return u;
}

// dE = G_b - G_a from the per-shell counter differences, and the decision.
template <int K, int NW, int PL>
__device__ __forceinline__ void finish_trial(uint8_t* box, int s, int sp, uint32_t a8, uint32_t b8,
                                             const uint32_t (&h)[kMaxShells][2], uint32_t ru, const Planes& P,
                                             int nA, const uint32_t* sA, const uint32_t* sB, unsigned& acc,
                                             long long& dsum) {
  const int a = (int)(a8 >> 3), b = (int)(b8 >> 3);
  int Ga = 0, Gb = 0;
#pragma unroll
  for (int p = 0; p < 4 * NW; p++) {
    int acc0 = 0, acc1 = 0, acc2 = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
#pragma unroll
      for (int w = 0; w < NW; w++) {
        const int d = (int)(h[k][w] ^ 0x80808080u);
        acc0 = dp4a_su(d, P.P[0][k][p][w], acc0);
        if (PL == 2) {
          acc1 = dp4a_ss(d, P.P[1][k][p][w], acc1);
        } else {
          acc1 = dp4a_su(d, P.P[1][k][p][w], acc1);
          acc2 = dp4a_ss(d, P.P[2][k][p][w], acc2);
        }
      }
    }
    const int G = acc0 + (acc1 << 8) + (acc2 << 16);
    Ga = (p == a) ? G : Ga;
    Gb = (p == b) ? G : Gb;
  }
  const int dE = Gb - Ga;
  if (metropolis_accept(dE, ru, sA, nA, sB)) {
    st_chk(box, s, 2 * SUB, kDbgBccBox, (uint8_t)b8);
    st_chk(box, sp, 2 * SUB, kDbgBccBox, (uint8_t)a8);
    acc++;
    dsum += dE;
  }
}

// dE = sum_k sum_c T_k[c] D_k[c] from the (a, b) row of V differences in
// shared memory (two 16-byte loads, eight dp4a), and the decision.
template <int K>
__device__ __forceinline__ void finish_trial_rows(uint8_t* box, int s, int sp, uint32_t a8, uint32_t b8,
                                                  const uint32_t (&h)[kMaxShells][2], uint32_t ru,
                                                  const uint32_t* s_rows, int nA, const uint32_t* sA,
                                                  const uint32_t* sB, unsigned& acc, long long& dsum) {
  const int a = (int)(a8 >> 3), b = (int)(b8 >> 3);
  const uint4* row = reinterpret_cast<const uint4*>(s_rows + (a * 4 + b) * 8);
  const uint4 lo = row[0], hi = row[1];
  const uint32_t Lw[4] = {lo.x, lo.y, lo.z, lo.w}, Hw[4] = {hi.x, hi.y, hi.z, hi.w};
  int dl = 0, dh = 0;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const int d = (int)(h[k][0] ^ 0x80808080u);
    dl = dp4a_su(d, Lw[k], dl);
    dh = dp4a_ss(d, Hw[k], dh);
  }
  const int dE = dl + (dh << 8);
  if (metropolis_accept(dE, ru, sA, nA, sB)) {
    st_chk(box, s, 2 * SUB, kDbgBccBox, (uint8_t)b8);
    st_chk(box, sp, 2 * SUB, kDbgBccBox, (uint8_t)a8);
    acc++;
    dsum += dE;
  }
}

// One tile pass: stage the tile of colour `tc` with index `jt` among the
// tiles of that colour (plus its 2-cell halo) into shared memory, run every
// intra-colour phase of the tile, write the tile and its 1-cell partner ring
// back, add the statistics.  Every thread of the CTA must call it.
// Shared memory: box (2 * SUB bytes), sA (nA words), sB (kNB words), s_stat[3].
// Shared-direction trial; defined where the offset table lives
// (smcx_sweep_bcc_dir.cu).
template <int B, int K, int NW, int PL>
__device__ void trial_shared_dir(uint8_t* box, int s, int dir, uint32_t ru, const Planes& P, const uint32_t* s_rows,
                                 int nA, const uint32_t* sA, const uint32_t* sB, unsigned& acc, unsigned& same,
                                 long long& dsum);

// Stage the tile and its 2-cell halo from 32-bit words of the site store, CW
// cells per word (4: one byte per cell, two 4-bit ids; 2: two int8 ids per
// cell).  Box column c of a row holds the cell at global x = t0x - 2 + c
// (periodic); the NWR words of a box row start at the multiple of CW at or
// below t0x - 2, and with nx a multiple of CW no word straddles the wrap.
// Lane l of a warp takes word l % NWR of row l / NWR of each group of RPS
// rows; warp w stages the planes w, w + nwarp, ..., and issues the loads of
// PLB planes (PLB * RS words per lane) before it unpacks them.
template <int CW>
__device__ __forceinline__ void stage_words(const LatDesc& D, uint8_t* box, const int* t0, int ex, int ey, int ez,
                                            int lane, int warp, int nwarp) {
  constexpr int h = 2;
  constexpr int NWR = (BOX + CW - 1) / CW + 1;  // words per box row (7 or 13)
  constexpr int RPS = 32 / NWR;                 // rows per warp step (4 or 2)
  constexpr int RS = BOX / RPS;                 // steps per plane (6 or 12)
  constexpr int PLB = 2;                        // planes per batch of loads
  constexpr int WPC = CW == 4 ? 1 : 2;          // bytes per cell
  const int nx = D.n[0], ny = D.n[1], nz = D.n[2];
  const int xs = t0[0] - h;
  const int r = xs & (CW - 1);  // xs - r is a multiple of CW (also for xs < 0)
  const int m = lane % NWR, ry = lane / NWR;
  const bool lane_ok = ry < RPS && CW * m - r < ex;
  int gw = (xs - r + CW * m) % nx;  // first cell of this lane's word
  gw += gw < 0 ? nx : 0;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(D.sites);
  const long long nword = (long long)nx * ny * nz * WPC / 4;
  for (int zb = warp; zb < ez; zb += nwarp * PLB) {
    uint32_t v[PLB][RS];
#pragma unroll
    for (int p = 0; p < PLB; p++) {
      const int zs = zb + p * nwarp;
      const long long zrow = zs < ez ? (long long)wrap_add(t0[2] - h, zs, nz) * ny : 0;
#pragma unroll
      for (int q = 0; q < RS; q++) {
        const int ys = RPS * q + ry;
        v[p][q] = 0;
        if (zs < ez && ys < ey && lane_ok) {
          const long long cell = (zrow + wrap_add(t0[1] - h, ys, ny)) * nx + gw;
          v[p][q] = ld_chk(words, cell * WPC / 4, nword, kDbgSite);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < PLB; p++) {
      const int zs = zb + p * nwarp;
#pragma unroll
      for (int q = 0; q < RS; q++) {
        const int ys = RPS * q + ry;
        if (zs < ez && ys < ey && lane_ok) {
          const int bi = zs * PP + ys * PX + CW * m - r;
#pragma unroll
          for (int j = 0; j < CW; j++) {
            const int c = CW * m + j - r;
            if (c >= 0 && c < ex) {
              const uint32_t s0 = CW == 4 ? (v[p][q] >> (8 * j)) & 15u : (v[p][q] >> (16 * j)) & 0xFFu;
              const uint32_t s1 = CW == 4 ? (v[p][q] >> (8 * j + 4)) & 15u : (v[p][q] >> (16 * j + 8)) & 0xFFu;
              st_chk(box, bi + j, 2 * SUB, kDbgBccStage, (uint8_t)(s0 << 3));
              st_chk(box, SUB + bi + j, 2 * SUB, kDbgBccStage, (uint8_t)(s1 << 3));
            }
          }
        }
      }
    }
  }
}

// Stage a tile (origin t0, extent ts) and its 2-cell halo into the box: from
// 32-bit words when nx is a multiple of the cells per word, else one lane per
// box column (ex <= BOX = 24 < 32), warp w the planes w, w + nwarp, ..., the
// loads of U rows of a plane issued before any is unpacked.  Every thread of
// the CTA takes part.
__device__ __forceinline__ void stage_box(const LatDesc& D, uint8_t* box, const int* t0, const int* ts, int lane,
                                          int warp, int nwarp) {
  constexpr int h = 2;
  const int ex = ts[0] + 2 * h, ey = ts[1] + 2 * h, ez = ts[2] + 2 * h;
  const int nx = D.n[0], ny = D.n[1], nz = D.n[2];
  const long long ncell = (long long)nx * ny * nz;
  if (D.storage == SMCX_INT8 ? (nx & 1) == 0 : (nx & 3) == 0) {
    if (D.storage == SMCX_INT8)
      stage_words<2>(D, box, t0, ex, ey, ez, lane, warp, nwarp);
    else
      stage_words<4>(D, box, t0, ex, ey, ez, lane, warp, nwarp);
  } else {
    constexpr int U = 8;
    const int gx = lane < ex ? wrap_add(t0[0] - h, lane, nx) : 0;
    for (int zs = warp; zs < ez; zs += nwarp) {
      const long long zrow = (long long)wrap_add(t0[2] - h, zs, nz) * ny;
      for (int ys0 = 0; ys0 < ey; ys0 += U) {
        uint32_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          v[u] = 0;
          if (ys < ey && lane < ex) {
            const long long cell = (zrow + wrap_add(t0[1] - h, ys, ny)) * nx + gx;
            v[u] = D.storage == SMCX_INT8
                       ? (uint32_t)ld_chk(reinterpret_cast<const uint16_t*>(D.sites), cell, ncell, kDbgSite)
                       : (uint32_t)ld_chk(D.sites, cell, ncell, kDbgSite);
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          if (ys < ey && lane < ex) {
            const uint32_t s0 = D.storage == SMCX_INT8 ? (v[u] & 0xFFu) : (v[u] & 15u);
            const uint32_t s1 = D.storage == SMCX_INT8 ? (v[u] >> 8) : (v[u] >> 4);
            const int bi = zs * PP + ys * PX + lane;
            st_chk(box, bi, 2 * SUB, kDbgBccStage, (uint8_t)(s0 << 3));
            st_chk(box, SUB + bi, 2 * SUB, kDbgBccStage, (uint8_t)(s1 << 3));
          }
        }
      }
    }
  }
}

// TL1: the acceptance tables are read from global memory through L1 instead
// of being copied into shared memory (sA, sB then point into D.thr), which
// frees 5 KB of shared memory per CTA.
template <int K, int NW, int PL, int SLOTS, int PROP = 0, bool TL1 = false>
__device__ __forceinline__ void bcc_tile_pass(const LatDesc& D, const Planes& Q, int tc, int jt,
                                              unsigned long long sweep, uint8_t* box, uint32_t* sA, uint32_t* sB,
                                              unsigned long long* s_stat) {
  __shared__ uint8_t s_dir[512];  // phase directions (shared-direction proposals)
  __shared__ __align__(16) uint32_t s_rows[PROP == 1 ? 128 : 4];  // V-difference rows (shared-direction)
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int ntc0 = D.nt[0] / 2, ntc1 = D.nt[1] / 2;
  const int jx = jt % ntc0, jy = (jt / ntc0) % ntc1, jz = jt / (ntc0 * ntc1);
  const int ti[3] = {2 * jx + (tc & 1), 2 * jy + ((tc >> 1) & 1), 2 * jz + ((tc >> 2) & 1)};
  int t0[3], ts[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int base = D.n[a] / D.nt[a], rem = D.n[a] % D.nt[a];
    ts[a] = base + (ti[a] < rem ? 1 : 0);
    t0[a] = ti[a] * base + min(ti[a], rem);
  }
  __syncthreads();  // the previous pass of this CTA is done with the tables
  if (tid < 3) s_stat[tid] = 0;
  if (TL1) {
    sA = const_cast<uint32_t*>(D.thr);
    sB = const_cast<uint32_t*>(D.thr) + kNA;
  } else {
    for (int i = tid; i < D.nA; i += nth) sA[i] = D.thr[i];
    for (int i = tid; i < kNB; i += nth) sB[i] = D.thr[kNA + i];
  }
  if (PROP == 1) {
    if (Q.rows)
      for (int i = tid; i < 128; i += nth) s_rows[i] = Q.R[i >> 3][i & 7];
    // per (sweep, tile, phase) (mode 1) or per (sweep, colour, block of two
    // tiles, phase) (mode 2)
    const unsigned tile = (unsigned)((ti[2] * D.nt[1] + ti[1]) * D.nt[0] + ti[0]);
    for (int pr = tid; pr < D.L * D.L * D.L; pr += nth) {
      const uint4 r = D.proposal == 2 ? block_direction_block(D.seed_lo, D.seed_hi, sweep, D.replica, tc,
                                                              (unsigned)jt >> 1, pr)
                                      : phase_direction_block(D.seed_lo, D.seed_hi, sweep, D.replica, tile, pr);
      st_chk(s_dir, 2 * pr, 512, kDbgBccDir, (uint8_t)(r.x >> 29));
      st_chk(s_dir, 2 * pr + 1, 512, kDbgBccDir, (uint8_t)(r.z >> 29));
    }
  }

  // stage tile + 2-cell halo
  constexpr int h = 2;
  const int nx = D.n[0], ny = D.n[1], nz = D.n[2];
  const long long ncell = (long long)nx * ny * nz;
  stage_box(D, box, t0, ts, lane, warp, nwarp);
  __syncthreads();

  // link-cell slots of this thread: q = tid + j * nth
  const int NQ = D.NQ, L = D.L;
  int qx[SLOTS], qy[SLOTS], qz[SLOTS];
  bool slot[SLOTS];
  // the bank-spreading lane order for the default shape (5^3 slots, 128
  // threads, one slot each); plain order otherwise
  const bool ordered = SLOTS == 1 && NQ == 5 && nth == 128;
#pragma unroll
  for (int j = 0; j < SLOTS; j++) {
    const int q = ordered ? (int)c_slot_order[tid] : tid + j * nth;
    qx[j] = q % NQ;
    qy[j] = (q / NQ) % NQ;
    qz[j] = q / (NQ * NQ);
    slot[j] = q < NQ * NQ * NQ;
  }
  unsigned acc = 0, same = 0;
  long long dsum = 0;
  for (int cz = 0; cz < L; cz++)
    for (int cy = 0; cy < L; cy++)
      for (int cx = 0; cx < L; cx++) {
        uint32_t keep_d[SLOTS], keep_u[SLOTS];
#pragma unroll
        for (int j = 0; j < SLOTS; j++) {
          const int xr = cx + L * qx[j], yr = cy + L * qy[j], zr = cz + L * qz[j];
          keep_d[j] = 0;
          keep_u[j] = 0;
          if (slot[j] && xr < ts[0] && yr < ts[1] && zr < ts[2]) {
            const unsigned long long cell =
                ((unsigned long long)(t0[2] + zr) * ny + (t0[1] + yr)) * nx + (t0[0] + xr);
            const uint4 rw = attempt_block(cell * 2, sweep, D.replica, D.seed_lo, D.seed_hi);
            keep_d[j] = rw.z;
            keep_u[j] = rw.w;
            const int s = (zr + h) * PP + (yr + h) * PX + (xr + h);
            if (PROP == 1)
              trial_shared_dir<0, K, NW, PL>(box, s, ld_chk(s_dir, ((cz * L + cy) * L + cx) * 2, 512, kDbgBccDir),
                                             rw.y, Q, s_rows, D.nA, sA, sB, acc, same, dsum);
            else
              trial<0, K, NW, PL>(box, s, rw.x, rw.y, Q, D.nA, sA, sB, acc, same, dsum);
          }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SLOTS; j++) {
          const int xr = cx + L * qx[j], yr = cy + L * qy[j], zr = cz + L * qz[j];
          if (slot[j] && xr < ts[0] && yr < ts[1] && zr < ts[2]) {
            const int s = (zr + h) * PP + (yr + h) * PX + (xr + h);
            if (PROP == 1)
              trial_shared_dir<1, K, NW, PL>(box, SUB + s,
                                             ld_chk(s_dir, ((cz * L + cy) * L + cx) * 2 + 1, 512, kDbgBccDir),
                                             keep_u[j], Q, s_rows, D.nA, sA, sB, acc, same, dsum);
            else
              trial<1, K, NW, PL>(box, SUB + s, keep_d[j], keep_u[j], Q, D.nA, sA, sB, acc, same, dsum);
          }
        }
        __syncthreads();
      }

  // write back tile + 1-cell partner ring: one lane per column (wx <= 22 <
  // 32), warp w the planes w, w + nwarp, ...
  const int wx = ts[0] + 2, wy = ts[1] + 2, wz = ts[2] + 2;
  const int gxw = lane < wx ? wrap_add(t0[0] - 1, lane, nx) : 0;
  for (int zw = warp; zw < wz; zw += nwarp) {
    const long long zrow = (long long)wrap_add(t0[2] - 1, zw, nz) * ny;
#pragma unroll 4
    for (int yw = 0; yw < wy; yw++) {
      if (lane < wx) {
        const long long cell = (zrow + wrap_add(t0[1] - 1, yw, ny)) * nx + gxw;
        const int bi = (zw + h - 1) * PP + (yw + h - 1) * PX + (lane + h - 1);
        const uint32_t s0 = ld_chk(box, bi, 2 * SUB, kDbgBccWrite) >> 3;
        const uint32_t s1 = ld_chk(box, SUB + bi, 2 * SUB, kDbgBccWrite) >> 3;
        if (D.storage == SMCX_INT8) {
          st_chk(D.sites, 2 * cell, 2 * ncell, kDbgSite, (uint8_t)s0);
          st_chk(D.sites, 2 * cell + 1, 2 * ncell, kDbgSite, (uint8_t)s1);
        } else {
          st_chk(D.sites, cell, ncell, kDbgSite, (uint8_t)(s0 | (s1 << 4)));
        }
      }
    }
  }

  add_stats_warp(s_stat, acc, same, dsum);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&D.stats[0], (unsigned long long)ts[0] * ts[1] * ts[2] * 2);
    atomicAdd(&D.stats[1], s_stat[0]);
    atomicAdd(&D.stats[2], s_stat[1]);
    atomicAdd(&D.stats[3], s_stat[2]);
  }
}

// Shared-memory bytes of one CTA running tile passes with tables of up to nA
// high-part entries.
__host__ __device__ constexpr size_t smem_bytes(int nA) { return 2 * SUB + (size_t)(nA + kNB) * 4; }


// Single-lattice sweep kernel: one CTA per tile of colour `tc`.
template <int K, int NW, int PL, int SLOTS, int PROP>
__global__ void __launch_bounds__(128, PROP == 1 ? 7 : 6) k_bcc_tile_sweep(const LatDesc D, const Planes Q, int tc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];
  uint8_t* box = smem;
  uint32_t* sA = reinterpret_cast<uint32_t*>(smem + 2 * SUB);
  uint32_t* sB = sA + D.nA;
  bcc_tile_pass<K, NW, PL, SLOTS, PROP, PROP == 1>(D, Q, tc, blockIdx.x, D.sweep, box, sA, sB, s_stat);
}

}  // namespace bccfast

template <int K, int NW, int PL, int SLOTS, int PROP = 0>
inline void launch_bcc(smcx_lattice* hd, bccfast::LatDesc& D, const bccfast::Planes& Q, int threads,
                       int64_t n_sweeps, int n_colours) {
  const size_t smem = PROP == 1 ? (size_t)2 * bccfast::SUB : bccfast::smem_bytes(D.nA);
  check_cuda(cudaFuncSetAttribute(bccfast::k_bcc_tile_sweep<K, NW, PL, SLOTS, PROP>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
             "bcc sweep smem attribute");
  if (PROP == 1)
    check_cuda(cudaFuncSetAttribute(bccfast::k_bcc_tile_sweep<K, NW, PL, SLOTS, PROP>,
                                    cudaFuncAttributePreferredSharedMemoryCarveout, 100),
               "bcc sweep carveout");
  const int grid = (D.nt[0] / 2) * (D.nt[1] / 2) * (D.nt[2] / 2);
  const unsigned long long first = D.sweep;
  for (int64_t s = 0; s < n_sweeps; s++) {
    D.sweep = first + (unsigned long long)s;
    for (int tc = 0; tc < n_colours; tc++)
      bccfast::k_bcc_tile_sweep<K, NW, PL, SLOTS, PROP><<<grid, threads, smem, hd->stream>>>(D, Q, tc);
  }
  check_cuda(cudaGetLastError(), "bcc sweep launch");
}

}  // namespace smcx
