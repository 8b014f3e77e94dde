// FCC tile pass specialised for throughput (pair model, M <= 8 species,
// K <= 3 shells, tiles up to 15 cells, link cells >= 3, one link-cell slot
// per thread).  Same trials, same order of phases, same Philox words and the
// same integer arithmetic as k_tile_sweep in smcx_sweep.cu: the result is
// bit-identical; only the data layout and the instruction mix differ.
//
//  * FCC sites are the even points (x + y + z even) of the half-unit cubic
//    grid.  Shared memory stores the box (tile + 2-cell halo, at most 38
//    half units per axis) with the site at half-unit box position (x, y, z)
//    in byte (x + y PXF + z PPF) / 2; PXF and PPF are odd, so the numerator
//    of every site is even and no byte is wasted.  A neighbour along the
//    lattice vector v is then at the constant offset (vx + vy PXF + vz PPF) /
//    2 from any site, whatever its sublattice: every load of the centre and
//    of the partner environment is one LDS with an immediate offset, and the
//    partner itself is one table entry away.
//  * Species are stored as 8 sigma; each neighbour adds 1 << (8 sigma) to a
//    per-shell register of byte counters (biased by 0x80), the s environment
//    adding and the s' environment subtracting; dE = G_b - G_a by dp4a
//    against the byte planes of V (finish_trial of the BCC pass).
//  * A thread owns one link-cell slot of the tile for the whole pass; the
//    Philox block of a site pair (sublattices 0/1 and 2/3 of a cell) is drawn
//    in the even phase and its second half used in the odd phase after it.
#include "smcx_bcc_tile.cuh"

namespace smcx {

namespace fccfast {

using bccfast::LatDesc;
using bccfast::Planes;

constexpr int H = 2;                     // halo cells
constexpr int TMAX = 15;                 // largest tile edge (cells)
constexpr int EXT = 2 * (TMAX + 2 * H);  // box edge in half units (38)
// Odd pitches (>= EXT and >= EXT * PXF) chosen by simulating the banks of a
// warp's 32 slot origins (link cell 3, 5^3 slots): every centre-environment
// load is one wavefront; the partner loads, scattered by the per-lane
// directions, are not.  No odd row pitch from 39 to 47 has such a plane
// pitch within 3000 bytes of the minimum; 49 / 1867 is the smallest box.
constexpr int PXF = 49;
constexpr int PPF = 1867;
static_assert(PXF % 2 == 1 && PPF % 2 == 1 && PXF > EXT - 1 && PPF >= EXT * PXF, "FCC box pitches");
constexpr int BOXB = ((EXT - 1) + (EXT - 1) * PXF + (EXT - 1) * PPF) / 2 + 1;  // bytes used
constexpr int BOX_BYTES = (BOXB + 15) / 16 * 16;

__host__ __device__ constexpr int hoff(int x, int y, int z) { return (x + y * PXF + z * PPF) / 2; }
// FCC basis (0,0,0), (1,1,0), (1,0,1), (0,1,1) in half units: offset of site b in its cell
__host__ __device__ constexpr int boff(int b) {
  return hoff((b == 1 || b == 2) ? 1 : 0, (b == 1 || b == 3) ? 1 : 0, (b == 2 || b == 3) ? 1 : 0);
}

// FCC lattice vectors of shells 1..3 (|v|^2 = 2, 4, 6 half units squared),
// shell-major, lexicographic inside a shell: the canonical order of the
// library and the oracle (shell-1 index = partner direction).
struct FVec {
  int x, y, z, k;
};
struct FTable {
  FVec v[42];
  int n;
};
__host__ __device__ constexpr FTable make_fvecs() {
  FTable t{};
  t.n = 0;
  for (int k = 0; k < 3; k++)
    for (int x = -2; x <= 2; x++)
      for (int y = -2; y <= 2; y++)
        for (int z = -2; z <= 2; z++) {
          if ((x + y + z) & 1) continue;
          if (x * x + y * y + z * z == 2 * (k + 1)) {
            t.v[t.n] = FVec{x, y, z, k};
            t.n++;
          }
        }
  return t;
}

template <int K, int NW, int SIGN>
__device__ __forceinline__ void gather(const uint8_t* box, int c, uint32_t (&h)[kMaxShells][2]) {
  constexpr FTable T = make_fvecs();
#pragma unroll
  for (int j = 0; j < T.n; j++) {
    const int k = T.v[j].k;
    if (k >= K) continue;
    const uint32_t v = ld_chk(box, c + hoff(T.v[j].x, T.v[j].y, T.v[j].z), BOX_BYTES, kDbgFccBox);
    if (NW <= 1) {
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

// dE = G_b - G_a with only the two V rows needed: the byte planes of V_k[p]
// are read from shared memory (sP [PL][K][8][NW]) at rows a and b, instead
// of forming G_p for every species slot in registers (8 NW K PL dp4a).  The
// FCC pass is bound by ALU issue, not by its shared-memory pipe, so the loads
// are the cheaper side.
template <int K, int NW, int PL>
__device__ __forceinline__ void finish_rows(uint8_t* box, int s, int sp, uint32_t a8, uint32_t b8,
                                            const uint32_t (&h)[kMaxShells][2], uint32_t ru, const uint32_t* sP,
                                            int nA, const uint32_t* sA, const uint32_t* sB, unsigned& acc,
                                            long long& dsum) {
  const int a = (int)(a8 >> 3), b = (int)(b8 >> 3);
  int ga0 = 0, ga1 = 0, ga2 = 0, gb0 = 0, gb1 = 0, gb2 = 0;
#pragma unroll
  for (int k = 0; k < K; k++) {
#pragma unroll
    for (int w = 0; w < NW; w++) {
      const int d = (int)(h[k][w] ^ 0x80808080u);
      const uint32_t* r0 = sP + ((0 * K + k) * 8) * NW + w;
      ga0 = bccfast::dp4a_su(d, r0[a * NW], ga0);
      gb0 = bccfast::dp4a_su(d, r0[b * NW], gb0);
      const uint32_t* r1 = sP + ((1 * K + k) * 8) * NW + w;
      if (PL == 2) {
        ga1 = bccfast::dp4a_ss(d, r1[a * NW], ga1);
        gb1 = bccfast::dp4a_ss(d, r1[b * NW], gb1);
      } else {
        ga1 = bccfast::dp4a_su(d, r1[a * NW], ga1);
        gb1 = bccfast::dp4a_su(d, r1[b * NW], gb1);
        const uint32_t* r2 = sP + ((2 * K + k) * 8) * NW + w;
        ga2 = bccfast::dp4a_ss(d, r2[a * NW], ga2);
        gb2 = bccfast::dp4a_ss(d, r2[b * NW], gb2);
      }
    }
  }
  const int dE = (gb0 + (gb1 << 8) + (gb2 << 16)) - (ga0 + (ga1 << 8) + (ga2 << 16));
  if (metropolis_accept(dE, ru, sA, nA, sB)) {
    st_chk(box, s, BOX_BYTES, kDbgFccBox, (uint8_t)b8);
    st_chk(box, sp, BOX_BYTES, kDbgFccBox, (uint8_t)a8);
    acc++;
    dsum += dE;
  }
}

// Six-bit counters (NW = 0, M <= 5): the box holds 6 sigma, each neighbour
// adds 1 << (6 sigma) to one word per shell (fields biased by 32; a count
// difference stays within +-24, so no field borrows from the next), and dE =
// sum_k sum_c (V_k[b][c] - V_k[a][c]) (field_kc - 32) from one row of the
// (a, b) table: K*5 differences and the bias term.  Rows sit 17 words apart
// in shared memory, so the lanes of a warp, whatever their (a, b), read
// distinct banks or the same word: every word load is one wavefront (16-byte
// loads of 16-word rows cost four or more).  Half the counter instructions
// of two byte-counter words.  The sum wraps modulo 2^32 like the int32 dE it
// ends as.
constexpr uint32_t kBias6 = 0x20820820u;  // 32 in each of the five 6-bit fields
struct Rows6 {
  int32_t r[25][16];  // r[a * 5 + b][k * 5 + c] = V_k[b][c] - V_k[a][c]; [15] = -32 sum
};
constexpr int kRowStride = 17;  // words between rows in shared memory
__device__ __forceinline__ int species6(uint32_t v6) { return (int)((v6 * 43u) >> 8); }  // v6 / 6, v6 <= 24

template <int K>
__device__ __forceinline__ void finish_six(uint8_t* box, int s, int sp, uint32_t a6, uint32_t b6,
                                           const uint32_t (&h)[kMaxShells][2], uint32_t ru, const int32_t* sR,
                                           int nA, const uint32_t* sA, const uint32_t* sB, unsigned& acc,
                                           long long& dsum) {
  const int32_t* row = sR + (species6(a6) * 5 + species6(b6)) * kRowStride;
  uint32_t e = (uint32_t)row[15];
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int c = 0; c < 5; c++) e += (uint32_t)row[k * 5 + c] * ((h[k][0] >> (6 * c)) & 63u);
  const int dE = (int)e;
  if (metropolis_accept(dE, ru, sA, nA, sB)) {
    st_chk(box, s, BOX_BYTES, kDbgFccBox, (uint8_t)b6);
    st_chk(box, sp, BOX_BYTES, kDbgFccBox, (uint8_t)a6);
    acc++;
    dsum += dE;
  }
}

template <int K, int NW, int PL>
__device__ __forceinline__ void trial(uint8_t* box, int s, uint32_t rd, uint32_t ru, const int* s_poff,
                                      const uint32_t* sP, const int32_t* sR, int nA, const uint32_t* sA,
                                      const uint32_t* sB, unsigned& acc, unsigned& same, long long& dsum) {
  const int dir = (int)__umulhi(rd, 12u);
  const int sp = s + s_poff[dir];
  const uint32_t a8 = ld_chk(box, s, BOX_BYTES, kDbgFccBox), b8 = ld_chk(box, sp, BOX_BYTES, kDbgFccBox);
  if (a8 == b8) {
    same++;
    return;
  }
  uint32_t h[kMaxShells][2];
#pragma unroll
  for (int k = 0; k < kMaxShells; k++) {
    h[k][0] = NW == 0 ? kBias6 : 0x80808080u;
    h[k][1] = 0x80808080u;
  }
  gather<K, NW, +1>(box, s, h);
  gather<K, NW, -1>(box, sp, h);
  // the s-s' bond is not part of either environment after the swap
  bccfast::add_one<NW == 0 ? 1 : NW>(h[0], b8, -1);
  bccfast::add_one<NW == 0 ? 1 : NW>(h[0], a8, +1);
  if constexpr (NW == 0)
    finish_six<K>(box, s, sp, a8, b8, h, ru, sR, nA, sA, sB, acc, dsum);
  else
    finish_rows<K, NW, PL>(box, s, sp, a8, b8, h, ru, sP, nA, sA, sB, acc, dsum);
}

// ---- shared-direction proposals (SMCX_PROPOSAL_TILE / _BLOCK) ------------
// One shell-1 direction p per (sweep, tile, intra colour): every lane of a
// phase swaps along the same vector, so the warp reads the union of the two
// environments at common offsets.  A site in shell k1 around s and k2 around
// s' = s + p adds one to counter k1 and subtracts one from counter k2; sites
// seeing both ends in the same shell cancel and are not read, nor are s and
// s' themselves (their bond is not part of either environment after the
// swap).  For 3 shells that leaves 50 of the 84 environment loads.  Entries
// are ordered by class (k1, k2), the same sequence of classes for every
// direction (the 12 directions are images of one another under the cubic
// group), so the shells are compile-time constants and only the box offsets,
// from a constant-memory row per direction, depend on p.
__host__ __device__ constexpr int fshell(int x, int y, int z) {
  const int r = x * x + y * y + z * z;
  return r == 2 ? 0 : r == 4 ? 1 : r == 6 ? 2 : -1;
}
constexpr int kFUnionMax = 64;
struct FUnion {
  int off[12][kFUnionMax];
  int k1[kFUnionMax], k2[kFUnionMax];
  int n;
  bool ok;
};
__host__ __device__ constexpr FUnion make_funion() {
  constexpr FTable T = make_fvecs();
  FUnion u{};
  u.ok = true;
  for (int d = 0; d < 12; d++) {
    const int px = T.v[d].x, py = T.v[d].y, pz = T.v[d].z;
    int n = 0;
    for (int a = -1; a < 3; a++)
      for (int b = -1; b < 3; b++) {
        if ((a < 0 && b < 0) || a == b) continue;
        // sites of shell a around s (a >= 0) seen in shell b around s'; or,
        // for a = -1, sites of shell b around s' outside the shells of s
        for (int j = 0; j < T.n; j++) {
          int x = 0, y = 0, z = 0;
          if (a >= 0) {
            if (T.v[j].k != a) continue;
            x = T.v[j].x;
            y = T.v[j].y;
            z = T.v[j].z;
            if (x == px && y == py && z == pz) continue;  // s'
            if (fshell(x - px, y - py, z - pz) != b) continue;
          } else {
            if (T.v[j].k != b) continue;
            x = T.v[j].x + px;
            y = T.v[j].y + py;
            z = T.v[j].z + pz;
            if ((x == 0 && y == 0 && z == 0) || fshell(x, y, z) >= 0) continue;  // s, or around s
          }
          if (n >= kFUnionMax) {
            u.ok = false;
            continue;
          }
          if (d == 0) {
            u.k1[n] = a;
            u.k2[n] = b;
          } else if (u.k1[n] != a || u.k2[n] != b) {
            u.ok = false;
          }
          u.off[d][n++] = hoff(x, y, z);
        }
      }
    if (d == 0) u.n = n;
    else if (n != u.n) u.ok = false;
  }
  return u;
}
static_assert(make_funion().ok, "FCC union classes differ between directions");
__constant__ FUnion c_funion = make_funion();

template <int K, int NW, int PL>
__device__ __forceinline__ void trial_dir(uint8_t* box, int s, int dir, uint32_t ru, const int* s_poff,
                                          const uint32_t* sP, const int32_t* sR, int nA, const uint32_t* sA,
                                          const uint32_t* sB, unsigned& acc, unsigned& same, long long& dsum) {
  static_assert(K == 3 && NW <= 1, "shared-direction FCC trials: 3 shells, one counter word");
  constexpr FUnion U = make_funion();
  const int sp = s + s_poff[dir];
  const uint32_t a8 = ld_chk(box, s, BOX_BYTES, kDbgFccBox), b8 = ld_chk(box, sp, BOX_BYTES, kDbgFccBox);
  if (a8 == b8) {
    same++;
    return;
  }
  uint32_t h[kMaxShells][2];
#pragma unroll
  for (int k = 0; k < kMaxShells; k++) {
    h[k][0] = NW == 0 ? kBias6 : 0x80808080u;
    h[k][1] = 0x80808080u;
  }
  const int* off = c_funion.off[dir];
#pragma unroll
  for (int i = 0; i < U.n; i++) {
    const uint32_t v = ld_chk(box, s + off[i], BOX_BYTES, kDbgFccBox);
    uint32_t one;
    asm("shl.b32 %0, 1, %1;" : "=r"(one) : "r"(v));
    if (U.k1[i] >= 0) h[U.k1[i]][0] += one;
    if (U.k2[i] >= 0) h[U.k2[i]][0] -= one;
  }
  if constexpr (NW == 0)
    finish_six<K>(box, s, sp, a8, b8, h, ru, sR, nA, sA, sB, acc, dsum);
  else
    finish_rows<K, NW, PL>(box, s, sp, a8, b8, h, ru, sP, nA, sA, sB, acc, dsum);
}

// Stage the tile and its 2-cell halo from 32-bit words of the site store,
// CPW cells per word (2: 16-bit cells of four 4-bit ids; 1: four int8 ids).
// Box column c of a row holds the cell at global x = t0x - 2 + c (periodic);
// the NWR words of a box row start at the multiple of CPW at or below
// t0x - 2, and with nx a multiple of CPW no word straddles the wrap.  Lane l
// of a warp takes word l % NWR of row l / NWR of each group of RPS rows; warp
// w stages the planes w, w + nwarp, ..., and issues the loads of PLB planes
// (PLB * RS words per lane) before it unpacks them.
template <int NW, int CPW>
__device__ __forceinline__ void stage_words(const LatDesc& D, uint8_t* box, const int (&t0)[3], int ex, int ey,
                                            int ez, int lane, int warp, int nwarp) {
  constexpr int BE = TMAX + 2 * H;               // box edge (cells)
  constexpr int NWR = CPW == 2 ? BE / 2 + 1 : BE;  // words per box row (10 or 19)
  constexpr int RPS = 32 / NWR;                  // rows per warp step (3 or 1)
  constexpr int RS = (BE + RPS - 1) / RPS;       // steps per plane (7 or 19)
  constexpr int PLB = CPW == 2 ? 2 : 1;          // planes per batch of loads
  const int nx = D.n[0], ny = D.n[1], nz = D.n[2];
  const int xs = t0[0] - H;
  const int r = xs & (CPW - 1);
  const int m = lane % NWR, ry = lane / NWR;
  const bool lane_ok = ry < RPS && CPW * m - r < ex;
  int gw = (xs - r + CPW * m) % nx;  // first cell of this lane's word
  gw += gw < 0 ? nx : 0;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(D.sites);
  const long long nword = (long long)nx * ny * nz / CPW;
  for (int zb = warp; zb < ez; zb += nwarp * PLB) {
    uint32_t v[PLB][RS];
#pragma unroll
    for (int p = 0; p < PLB; p++) {
      const int zs = zb + p * nwarp;
      const long long zrow = zs < ez ? (long long)wrap_add(t0[2] - H, zs, nz) * ny : 0;
#pragma unroll
      for (int q = 0; q < RS; q++) {
        const int ys = RPS * q + ry;
        v[p][q] = 0;
        if (zs < ez && ys < ey && lane_ok) {
          const long long cell = (zrow + wrap_add(t0[1] - H, ys, ny)) * nx + gw;
          v[p][q] = ld_chk(words, cell / CPW, nword, kDbgSite);
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
#pragma unroll
          for (int j = 0; j < CPW; j++) {
            const int c = CPW * m + j - r;
            if (c >= 0 && c < ex) {
              const uint32_t cv = CPW == 2 ? (v[p][q] >> (16 * j)) & 0xFFFFu : v[p][q];
              const int base = hoff(2 * c, 2 * ys, 2 * zs);
#pragma unroll
              for (int b = 0; b < 4; b++) {
                const uint32_t sp = CPW == 2 ? (cv >> (4 * b)) & 15u : (cv >> (8 * b)) & 0xFFu;
                st_chk(box, base + boff(b), BOX_BYTES, kDbgFccBox, (uint8_t)(NW == 0 ? sp * 6 : sp << 3));
              }
            }
          }
        }
      }
    }
  }
}

// box, partner offsets (16 ints), six-bit rows (25 x 17 words), plane rows
// (3 x 3 x 8 x 2 words), sA, sB
constexpr int kPlaneWords = 3 * 3 * 8 * 2;
constexpr int kRowWords = 25 * 17;
__host__ __device__ constexpr size_t smem_bytes(int nA) {
  return BOX_BYTES + 16 * 4 + kRowWords * 4 + kPlaneWords * 4 + (size_t)(nA + kNB) * 4;
}

// Five CTAs per SM: the box and its tables (42.8 KB) allow no sixth, so the
// launch bounds leave the kernel 102 registers (it takes 96).
template <int K, int NW, int PL, int PROP = 0>
__global__ void __launch_bounds__(128, 5) k_fcc_tile_sweep(const LatDesc D, const Planes Q, const Rows6 R, int tc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];
  __shared__ uint8_t s_dir[PROP ? 512 : 4];  // phase directions (shared-direction proposals)
  uint8_t* box = smem;
  int* s_poff = reinterpret_cast<int*>(smem + BOX_BYTES);
  int32_t* sR = s_poff + 16;
  uint32_t* sP = reinterpret_cast<uint32_t*>(sR + kRowWords);
  uint32_t* sA = sP + kPlaneWords;
  uint32_t* sB = sA + D.nA;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int jt = blockIdx.x;
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
  if (tid < 3) s_stat[tid] = 0;
  if constexpr (NW > 0) {
    for (int i = tid; i < PL * K * 8 * NW; i += nth) {
      const int w = i % NW, p = (i / NW) % 8, k = (i / (NW * 8)) % K, j = i / (NW * 8 * K);
      sP[i] = Q.P[j][k][p][w];
    }
  } else {
    for (int i = tid; i < 25 * 16; i += nth) sR[(i / 16) * kRowStride + i % 16] = R.r[i / 16][i % 16];
  }
  for (int i = tid; i < D.nA; i += nth) sA[i] = D.thr[i];
  for (int i = tid; i < kNB; i += nth) sB[i] = D.thr[kNA + i];
  if constexpr (PROP != 0) {
    // per (sweep, tile, intra colour ic) (mode 1) or per (sweep, colour,
    // block of two tiles, ic) (mode 2): one Philox block per ic pair pr =
    // ic >> 1, word 0 for even ic, word 2 for odd ic
    const unsigned tile = (unsigned)((ti[2] * D.nt[1] + ti[1]) * D.nt[0] + ti[0]);
    for (int pr = tid; pr < 2 * D.L * D.L * D.L; pr += nth) {
      const uint4 r = D.proposal == 2 ? block_direction_block(D.seed_lo, D.seed_hi, D.sweep, D.replica, tc,
                                                              (unsigned)jt >> 1, pr)
                                      : phase_direction_block(D.seed_lo, D.seed_hi, D.sweep, D.replica, tile, pr);
      st_chk(s_dir, 2 * pr, 512, kDbgBccDir, (uint8_t)__umulhi(r.x, 12u));
      st_chk(s_dir, 2 * pr + 1, 512, kDbgBccDir, (uint8_t)__umulhi(r.z, 12u));
    }
  }
  if (tid < 12) {
    constexpr FTable T = make_fvecs();
    int o = 0;
#pragma unroll
    for (int d = 0; d < 12; d++)
      if (d == tid) o = hoff(T.v[d].x, T.v[d].y, T.v[d].z);
    s_poff[tid] = o;
  }

  // stage tile + 2-cell halo
  const int ex = ts[0] + 2 * H, ey = ts[1] + 2 * H, ez = ts[2] + 2 * H;
  const int nx = D.n[0], ny = D.n[1], nz = D.n[2];
  if (D.storage == SMCX_INT8)
    stage_words<NW, 1>(D, box, t0, ex, ey, ez, lane, warp, nwarp);
  else if ((nx & 1) == 0)
    stage_words<NW, 2>(D, box, t0, ex, ey, ez, lane, warp, nwarp);
  else {
    // odd x extent, 16-bit cells: one box column (cell x) per lane, warp w
    // the planes w, w + nwarp, ..., 8 rows of global loads in flight per lane
    constexpr int U = 8;
    const int gx = lane < ex ? wrap_add(t0[0] - H, lane, nx) : 0;
    for (int zs = warp; zs < ez; zs += nwarp) {
      const long long zrow = (long long)wrap_add(t0[2] - H, zs, nz) * ny;
      for (int ys0 = 0; ys0 < ey; ys0 += U) {
        uint32_t v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          v[u] = 0;
          if (ys < ey && lane < ex) {
            const long long cell = (zrow + wrap_add(t0[1] - H, ys, ny)) * nx + gx;
            v[u] = (uint32_t)(*reinterpret_cast<const uint16_t*>(D.sites + 2 * cell));
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          if (ys < ey && lane < ex) {
            const int base = hoff(2 * lane, 2 * ys, 2 * zs);
#pragma unroll
            for (int b = 0; b < 4; b++) {
              const uint32_t sp = (v[u] >> (4 * b)) & 15u;
              st_chk(box, base + boff(b), BOX_BYTES, kDbgFccBox, (uint8_t)(NW == 0 ? sp * 6 : sp << 3));
            }
          }
        }
      }
    }
  }
  __syncthreads();

  // this thread's link-cell slot
  const int NQ = D.NQ, L = D.L;
  const int qx = tid % NQ, qy = (tid / NQ) % NQ, qz = tid / (NQ * NQ);
  const bool slot = tid < NQ * NQ * NQ;
  unsigned acc = 0, same = 0;
  long long dsum = 0;
  for (int cz = 0; cz < L; cz++)
    for (int cy = 0; cy < L; cy++)
      for (int cx = 0; cx < L; cx++) {
        const int xr = cx + L * qx, yr = cy + L * qy, zr = cz + L * qz;
        const bool here = slot && xr < ts[0] && yr < ts[1] && zr < ts[2];
        const int cbase = hoff(2 * (xr + H), 2 * (yr + H), 2 * (zr + H));
        const unsigned long long cell = ((unsigned long long)(t0[2] + zr) * ny + (t0[1] + yr)) * nx + (t0[0] + xr);
#pragma unroll
        for (int pr = 0; pr < 2; pr++) {
          // sublattices 2 pr and 2 pr + 1 share the Philox block of pair cell*2 + pr
          uint4 rw = make_uint4(0, 0, 0, 0);
          const int ic = (((cz * L + cy) * L + cx) * 4) + 2 * pr;
          if (here) {
            rw = attempt_block(cell * 4 + 2 * pr, D.sweep, D.replica, D.seed_lo, D.seed_hi);
            if constexpr (PROP != 0)
              trial_dir<K, NW, PL>(box, cbase + boff(2 * pr), ld_chk(s_dir, ic, 512, kDbgBccDir), rw.y, s_poff, sP,
                                   sR, D.nA, sA, sB, acc, same, dsum);
            else
              trial<K, NW, PL>(box, cbase + boff(2 * pr), rw.x, rw.y, s_poff, sP, sR, D.nA,
                               sA, sB, acc, same, dsum);
          }
          __syncthreads();
          if (here) {
            if constexpr (PROP != 0)
              trial_dir<K, NW, PL>(box, cbase + boff(2 * pr + 1), ld_chk(s_dir, ic + 1, 512, kDbgBccDir), rw.w,
                                   s_poff, sP, sR, D.nA, sA, sB, acc, same, dsum);
            else
              trial<K, NW, PL>(box, cbase + boff(2 * pr + 1), rw.z, rw.w, s_poff,
                               sP, sR, D.nA, sA, sB, acc, same, dsum);
          }
          __syncthreads();
        }
      }

  // write back tile + 1-cell partner ring: one lane per column (wx <= 17 <
  // 32), warp w the planes w, w + nwarp, ...
  const int wx = ts[0] + 2, wy = ts[1] + 2, wz = ts[2] + 2;
  const int gxw = lane < wx ? wrap_add(t0[0] - 1, lane, nx) : 0;
  for (int zw = warp; zw < wz; zw += nwarp) {
    const long long zrow = (long long)wrap_add(t0[2] - 1, zw, nz) * ny;
#pragma unroll 4
    for (int yw = 0; yw < wy; yw++) {
      if (lane < wx) {
        const long long cell = (zrow + wrap_add(t0[1] - 1, yw, ny)) * nx + gxw;
        const int base = hoff(2 * (lane + H - 1), 2 * (yw + H - 1), 2 * (zw + H - 1));
        uint32_t s4[4];
#pragma unroll
        for (int b = 0; b < 4; b++) {
          const uint32_t v = ld_chk(box, base + boff(b), BOX_BYTES, kDbgFccBox);
          s4[b] = NW == 0 ? (uint32_t)species6(v) : v >> 3;
        }
        if (D.storage == SMCX_INT8) {
          *reinterpret_cast<uint32_t*>(D.sites + 4 * cell) = s4[0] | (s4[1] << 8) | (s4[2] << 16) | (s4[3] << 24);
        } else {
          *reinterpret_cast<uint16_t*>(D.sites + 2 * cell) =
              (uint16_t)(s4[0] | (s4[1] << 4) | (s4[2] << 8) | (s4[3] << 12));
        }
      }
    }
  }

  add_stats_warp(s_stat, acc, same, dsum);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&D.stats[0], (unsigned long long)ts[0] * ts[1] * ts[2] * 4);
    atomicAdd(&D.stats[1], s_stat[0]);
    atomicAdd(&D.stats[2], s_stat[1]);
    atomicAdd(&D.stats[3], s_stat[2]);
  }
}

}  // namespace fccfast

int build_planes(const smcx_lattice* hd, bccfast::Planes* Q, int min_planes);

// FCC pair model, M <= 8, K <= 3, |V| < 2^23, a tiled schedule with tiles of
// at most 15 cells and link cells of at least 3 (one slot of at most 5^3 per
// thread of a 128-thread CTA), 16-byte aligned store.  Shared-direction
// proposals: 3 shells and one counter word (M <= 5; M <= 4 with |V| < 2^15).
bool fcc_fast_usable(const smcx_lattice* hd) {
  const smcx_sched& sc = hd->sched;
  if (hd->kind != kFCC || hd->M > kMaxSweepM || !hd->have_epi || !hd->Wq.empty()) return false;
  if (hd->shells.K > 3) return false;
  if (hd->proposal != SMCX_PROPOSAL_SITE) {
    if (hd->shells.K != 3 || hd->M > 5) return false;
    if (hd->M == 5) {
      // six-bit counters: every field difference fits
    } else {
      for (int32_t v : hd->V)
        if (v >= 32768 || v <= -32768) return false;  // one counter word, two byte planes
    }
  }
  if (sc.L < 3 || sc.nt[0] < 2 || sc.nt[1] < 2 || sc.nt[2] < 2) return false;
  if (halo_cells(hd->shells) != 2 || ring_cells(hd->shells) != 1) return false;
  if (reinterpret_cast<uintptr_t>(hd->d_sites) % 4 != 0) return false;
  for (int32_t v : hd->V)
    if (v >= (1 << 23) || v <= -(1 << 23)) return false;
  int nq = 0;
  for (int a = 0; a < 3; a++) {
    const int tmax = (hd->n[a] + sc.nt[a] - 1) / sc.nt[a];
    if (tmax > fccfast::TMAX) return false;
    nq = std::max(nq, (tmax + sc.L - 1) / sc.L);
  }
  return nq * nq * nq <= 128;
}

void sweep_fcc_fast(smcx_lattice* hd, int nA, uint64_t seed, int64_t n_sweeps, int n_colours) {
  bccfast::LatDesc D;
  memset(&D, 0, sizeof(D));
  const smcx_sched& sc = hd->sched;
  D.sites = hd->d_sites;
  D.thr = hd->d_thr;
  D.stats = hd->d_stats;
  int nq = 0;
  for (int a = 0; a < 3; a++) {
    D.n[a] = hd->n[a];
    D.nt[a] = sc.nt[a];
    nq = std::max(nq, ((hd->n[a] + sc.nt[a] - 1) / sc.nt[a] + sc.L - 1) / sc.L);
  }
  D.L = sc.L;
  D.NQ = nq;
  D.nA = nA;
  D.storage = hd->storage;
  D.replica = hd->replica;
  D.seed_lo = (uint32_t)seed;
  D.seed_hi = (uint32_t)(seed >> 32);
  D.M = hd->M;
  D.proposal = hd->proposal;
  bccfast::Planes Q;
  const int K = hd->shells.K;
  const int PL = build_planes(hd, &Q, K == 3 ? 2 : 3);
  // counters: one byte-counter word (3 shells, M <= 4), six-bit fields in one
  // word (M <= 5), else two byte-counter words
  const int M = hd->M;
  const int NW = (K == 3 && M <= 4) ? 1 : M <= 5 ? 0 : 2;
  fccfast::Rows6 R;
  memset(&R, 0, sizeof(R));
  if (NW == 0)
    for (int a = 0; a < M; a++)
      for (int b = 0; b < M; b++) {
        int32_t* r = R.r[a * 5 + b];
        uint32_t sum = 0;
        for (int k = 0; k < K; k++)
          for (int c = 0; c < M; c++) {
            r[k * 5 + c] = hd->V[((size_t)k * M + b) * M + c] - hd->V[((size_t)k * M + a) * M + c];
            sum += (uint32_t)r[k * 5 + c];
          }
        r[15] = (int32_t)(0u - 32u * sum);
      }
  const size_t smem = fccfast::smem_bytes(nA);
  const int grid = (D.nt[0] / 2) * (D.nt[1] / 2) * (D.nt[2] / 2);
  auto run = [&](auto kern) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "fcc sweep smem attribute");
    const unsigned long long first = hd->sweep_cum;
    for (int64_t s = 0; s < n_sweeps; s++) {
      D.sweep = first + (unsigned long long)s;
      for (int tc = 0; tc < n_colours; tc++) kern<<<grid, 128, smem, hd->stream>>>(D, Q, R, tc);
    }
  };
  if (D.proposal != 0) {
    // shared-direction proposals (fcc_fast_usable: 3 shells, one counter word)
    if (NW == 0) run(fccfast::k_fcc_tile_sweep<3, 0, 0, 1>);
    else if (NW == 1 && PL == 2) run(fccfast::k_fcc_tile_sweep<3, 1, 2, 1>);
    else fail(SMCX_E_UNSUPPORTED, "shared-direction FCC kernel: 3 shells, M <= 5");
  } else if (NW == 0) {
    if (K == 3) run(fccfast::k_fcc_tile_sweep<3, 0, 0>);
    else if (K == 2) run(fccfast::k_fcc_tile_sweep<2, 0, 0>);
    else run(fccfast::k_fcc_tile_sweep<1, 0, 0>);
  } else if (K == 3) {
    if (NW == 1) {
      if (PL == 2) run(fccfast::k_fcc_tile_sweep<3, 1, 2>);
      else run(fccfast::k_fcc_tile_sweep<3, 1, 3>);
    } else {
      if (PL == 2) run(fccfast::k_fcc_tile_sweep<3, 2, 2>);
      else run(fccfast::k_fcc_tile_sweep<3, 2, 3>);
    }
  } else if (K == 2) {
    run(fccfast::k_fcc_tile_sweep<2, 2, 3>);
  } else {
    run(fccfast::k_fcc_tile_sweep<1, 2, 3>);
  }
  check_cuda(cudaGetLastError(), "fcc sweep launch");
}

}  // namespace smcx
