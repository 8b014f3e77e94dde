// Sweeps of the qSRO model (Method "The EPI and qSRO model", Eq.
// quadratic_local_SRO), integer form: the pair terms plus, for every site i,
// sum_k W_k[s_i] n_k(i)^2, n_k(i) = number of shell-k neighbours of i with
// i's own species (the same-element pair fraction times z_k; W carries the
// 1/z_k^2 and is in 0.01 meV).
//
// The paper computes such energy changes by adding up the local energies of
// every site in the LIZ.  Here a trial swapping a (at s) and b (at s')
// computes the change exactly from what actually moves:
//  * the pair part, as in the pair-model kernels;
//  * s and s' themselves: their same-species counts before (species a at s,
//    b at s') and after (b at s, a at s'), from the two environments that
//    the pair part reads anyway;
//  * every other site i of the two environments whose species c is a or b
//    and that sees s in shell k1 and s' in shell k2 with k1 != k2: n_k1(i)
//    changes by d1 = +1 (c = b) or -1 (c = a) and n_k2(i) by -d1, so its term
//    changes by W_k[c] (2 d n_k(i) + 1) for those shells.  Sites of other
//    species, or seeing both ends in the same shell, do not change.
// Two kernels get n_k(i):
//  * k_qsro_fcc_n (FCC, 2 or 3 shells, tiles of 3 to 20 cells) keeps every
//    site's counts beside its species (a device array written once per sweep
//    call, a 16-bit shared-memory box during a tile pass) and updates them
//    on accepted swaps, so a count is one load;
//  * k_tile_sweep_qsro (BCC, and FCC with larger tiles) counts i's own
//    shell-k neighbours in shared memory.
// k2 (the shell of s' - i for i = s + v) and whether s' + v lies in the
// environment of s are per-direction tables (built on the host for the
// generic kernel, at compile time for the FCC one).
//
// The trial reads R1 + 2 R_K around its centre, so the schedule uses the
// larger link cell and halo of this model (FCC with 3 shells: L >= 4, the
// paper's 4x4x4); tiles run concurrently exactly as in k_tile_sweep.
#include <algorithm>

#include "smcx_device.cuh"

namespace smcx {

struct QsroTables {
  int32_t W[kMaxShells * kMaxSweepM];  // W[k][c]
  signed char k2[kMaxZ1][kMaxVec];      // shell of (p_dir - v_j); -1 outside K shells; -2 when zero
  signed char in_s[kMaxZ1][kMaxVec];    // 1 when p_dir + v_j is 0 or inside the K shells
  signed char sub[4][kMaxVec];          // sublattice of the site centre_b + v_j
  unsigned char start[kMaxShells + 1];  // first vector of each shell
};

// NT threads per CTA: 128 when a phase of the tile has at most 128 trials
// (20-cell tiles, L = 4: 125), else 256; registers capped for 512 threads/SM.
template <int KIND, int K, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_tile_sweep_qsro(const SweepParams P, const QsroTables Q) {
  constexpr int m = cell_sites(KIND);
  constexpr int NV = vec_count(KIND, K);
  constexpr int Z1 = shell_size(KIND, 0);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];
  __shared__ int32_t s_wq[kMaxShells * kMaxSweepM];
  __shared__ signed char s_k2[kMaxZ1 * NV], s_ins[kMaxZ1 * NV], s_sub[4 * NV];
  __shared__ int s_start[kMaxShells + 1];

  const int tid = threadIdx.x, nth = blockDim.x;
  const int M = P.M, KM = K * P.M, MM = P.M * P.M;
  const int nW = MM * KM + MM;
  int32_t* s_w = reinterpret_cast<int32_t*>(smem);
  uint32_t* s_A = reinterpret_cast<uint32_t*>(s_w + nW);
  uint32_t* s_B = s_A + P.nA;
  int* s_off = reinterpret_cast<int*>(s_B + kNB);
  int* s_poff = s_off + m * NV;
  int* s_psub = s_poff + m * Z1;
  int8_t* box = reinterpret_cast<int8_t*>(s_psub + m * Z1);

  int bid = blockIdx.x;
  const int jx = bid % P.ntc[0];
  bid /= P.ntc[0];
  const int jy = bid % P.ntc[1];
  const int jz = bid / P.ntc[1];
  const int ti[3] = {2 * jx + (P.tc & 1), 2 * jy + ((P.tc >> 1) & 1), 2 * jz + ((P.tc >> 2) & 1)};
  int t0[3], ts[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int base = P.n[a] / P.nt[a], rem = P.n[a] % P.nt[a];
    ts[a] = base + (ti[a] < rem ? 1 : 0);
    t0[a] = ti[a] * base + min(ti[a], rem);
  }

  if (tid < 3) s_stat[tid] = 0;
  for (int i = tid; i < nW; i += nth) s_w[i] = P.wtab[i];
  for (int i = tid; i < P.nA; i += nth) s_A[i] = P.thr[i];
  for (int i = tid; i < kNB; i += nth) s_B[i] = P.thr[kNA + i];
  for (int i = tid; i < m * NV; i += nth) s_off[i] = P.off[i / NV][i % NV];
  for (int i = tid; i < m * Z1; i += nth) {
    s_poff[i] = P.poff[i / Z1][i % Z1];
    s_psub[i] = P.psub[i / Z1][i % Z1];
  }
  for (int i = tid; i < KM; i += nth) s_wq[i] = Q.W[i];
  for (int i = tid; i < Z1 * NV; i += nth) {
    s_k2[i] = Q.k2[i / NV][i % NV];
    s_ins[i] = Q.in_s[i / NV][i % NV];
  }
  for (int i = tid; i < m * NV; i += nth) s_sub[i] = Q.sub[i / NV][i % NV];
  for (int i = tid; i <= K; i += nth) s_start[i] = Q.start[i];

  const int h = P.h;
  stage_generic<m>(P, box, t0, ts, h);
  __syncthreads();

  // same-species neighbours of box site i (sublattice bi) in shell k
  auto count = [&](int i, int bi, int k, int c) {
    int n = 0;
    const int* off = s_off + bi * NV;
    for (int j = s_start[k]; j < s_start[k + 1]; j++) n += (box[i + off[j]] == c);
    return n;
  };

  unsigned long long acc = 0, same = 0;
  long long dsum = 0;
  const int L = P.L;
  const int nic = L * L * L * m;
  for (int ic = 0; ic < nic; ic++) {
    const int b = ic % m, lc = ic / m;
    const int cx = lc % L, cy = (lc / L) % L, cz = lc / (L * L);
    const int nxp = ts[0] > cx ? (ts[0] - cx + L - 1) / L : 0;
    const int nyp = ts[1] > cy ? (ts[1] - cy + L - 1) / L : 0;
    const int nzp = ts[2] > cz ? (ts[2] - cz + L - 1) / L : 0;
    const int np = nxp * nyp * nzp;
    for (int i = tid; i < np; i += nth) {
      const int ix = i % nxp, r = i / nxp, iy = r % nyp, iz = r / nyp;
      const int xr = cx + L * ix, yr = cy + L * iy, zr = cz + L * iz;
      const int s = (((zr + h) * P.BY + (yr + h)) * P.BX + (xr + h)) * m + b;
      const unsigned long long gid =
          ((((unsigned long long)(t0[2] + zr)) * P.n[1] + (t0[1] + yr)) * P.n[0] + (t0[0] + xr)) * m + b;
      const uint4 rw = attempt_block(gid, P.sweep, P.replica, P.seed_lo, P.seed_hi);
      const uint32_t rd = (gid & 1) ? rw.z : rw.x;
      const uint32_t ru = (gid & 1) ? rw.w : rw.y;
      const int dir = (int)__umulhi(rd, (uint32_t)Z1);
      const int sp = s + s_poff[b * Z1 + dir];
      const int bp = s_psub[b * Z1 + dir];
      const int sa = box[s], sb = box[sp];
      if (sa == sb) {
        same++;
        continue;
      }
      // pair part, and the same-species counts of s and s'
      const int32_t* W = s_w + (sa * M + sb) * KM;
      int dE = s_w[MM * KM + sa * M + sb];
      int na_s[K], nb_s[K], na_p[K], nb_p[K];
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
          na_s[k] = nb_s[k] = 0;
#pragma unroll
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const int t = s + s_off[b * NV + j];
            const int c = box[t];
            dE += W[k * M + c];
            if (t != sp) {
              na_s[k] += (c == sa);
              nb_s[k] += (c == sb);
            }
          }
        }
      }
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
          na_p[k] = nb_p[k] = 0;
#pragma unroll
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const int t = sp + s_off[bp * NV + j];
            const int c = box[t];
            dE -= W[k * M + c];
            if (t != s) {
              na_p[k] += (c == sa);
              nb_p[k] += (c == sb);
            }
          }
        }
      }
      // quadratic terms of s and s' (before: a at s, b at s'; after: swapped)
#pragma unroll
      for (int k = 0; k < K; k++)
        dE += s_wq[k * M + sb] * (nb_s[k] * nb_s[k] - nb_p[k] * nb_p[k]) +
              s_wq[k * M + sa] * (na_p[k] * na_p[k] - na_s[k] * na_s[k]);
      // other sites of the environment of s
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const int t = s + s_off[b * NV + j];
            const int c = box[t];
            if (c != sa && c != sb) continue;
            const int k2 = s_k2[dir * NV + j];
            if (k2 == -2 || k2 == k) continue;  // t is s', or sees s and s' in one shell
            const int bt = s_sub[b * NV + j];
            const int d1 = (c == sb) ? 1 : -1;
            dE += s_wq[k * M + c] * (2 * d1 * count(t, bt, k, c) + 1);
            if (k2 >= 0) dE += s_wq[k2 * M + c] * (-2 * d1 * count(t, bt, k2, c) + 1);
          }
        }
      }
      // sites that see only s'
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            if (s_ins[dir * NV + j]) continue;
            const int t = sp + s_off[bp * NV + j];
            const int c = box[t];
            if (c != sa && c != sb) continue;
            const int d2 = (c == sb) ? -1 : 1;
            dE += s_wq[k * M + c] * (2 * d2 * count(t, s_sub[bp * NV + j], k, c) + 1);
          }
        }
      }
      if (metropolis_accept(dE, ru, s_A, P.nA, s_B)) {
        box[s] = (int8_t)sb;
        box[sp] = (int8_t)sa;
        acc++;
        dsum += dE;
      }
    }
    __syncthreads();
  }

  write_back_generic<m>(P, box, t0, ts, h, P.ring);

  add_stats_warp(s_stat, (unsigned)acc, (unsigned)same, dsum);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&P.stats[0], (unsigned long long)ts[0] * ts[1] * ts[2] * m);
    atomicAdd(&P.stats[1], s_stat[0]);
    atomicAdd(&P.stats[2], s_stat[1]);
    atomicAdd(&P.stats[3], s_stat[2]);
  }
}

// ---------------------------------------------------------------------------
// FCC even-point species box (used to count every site's same-species
// neighbours at the start of a sweep call): the FCC sites are the even
// points of the half-unit grid, stored at byte (x + y QPX + z QPP) / 2 of a
// box of QEXT half units per axis (tile <= 20 cells + 3-cell halo), so a
// neighbour along v is at a constant offset from any site and a shell count
// is an unrolled run of immediate-offset loads.
// ---------------------------------------------------------------------------
namespace qfcc {
constexpr int H = 3;
constexpr int TMAX = 20;
constexpr int QEXT = 2 * (TMAX + 2 * H);  // 52
constexpr int QPX = QEXT + 1;             // 53, odd
constexpr int QPP = QPX * QEXT + 1;       // 2757, odd
constexpr int BOXB = ((QEXT - 1) + (QEXT - 1) * QPX + (QEXT - 1) * QPP) / 2 + 1;
constexpr int BOX_BYTES = (BOXB + 15) / 16 * 16;
__host__ __device__ constexpr int hoff(int x, int y, int z) { return (x + y * QPX + z * QPP) / 2; }
__host__ __device__ constexpr int boff(int b) {
  return hoff((b == 1 || b == 2) ? 1 : 0, (b == 1 || b == 3) ? 1 : 0, (b == 2 || b == 3) ? 1 : 0);
}
struct QVec {
  int x, y, z, k;
};
struct QTable {
  QVec v[42];
  int n;
  int start[4];
};
__host__ __device__ constexpr QTable make_qvecs() {
  QTable t{};
  t.n = 0;
  for (int k = 0; k < 3; k++) {
    t.start[k] = t.n;
    for (int x = -2; x <= 2; x++)
      for (int y = -2; y <= 2; y++)
        for (int z = -2; z <= 2; z++) {
          if ((x + y + z) & 1) continue;
          if (x * x + y * y + z * z == 2 * (k + 1)) {
            t.v[t.n] = QVec{x, y, z, k};
            t.n++;
          }
        }
  }
  t.start[3] = t.n;
  return t;
}
// same-species (c) neighbours of box site t in shell KS
template <int KS>
__device__ __forceinline__ int count_shell(const uint8_t* box, int t, int c) {
  constexpr QTable T = make_qvecs();
  int n = 0;
#pragma unroll
  for (int j = T.start[KS]; j < T.start[KS + 1]; j++) n += (box[t + hoff(T.v[j].x, T.v[j].y, T.v[j].z)] == c);
  return n;
}
// Stage tile + 3-cell halo (species bytes at the even points): one box
// column per lane, warp w the planes w, w + nwarp, ..., the loads of 8 rows
// of a plane issued before any is unpacked; every thread of the CTA takes
// part.
__device__ __forceinline__ void stage_box(const SweepParams& P, uint8_t* box, const int (&t0)[3], const int (&ts)[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ex = ts[0] + 2 * H, ey = ts[1] + 2 * H, ez = ts[2] + 2 * H;
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
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
          v[u] = P.storage == SMCX_INT8 ? *reinterpret_cast<const uint32_t*>(P.sites + 4 * cell)
                                        : (uint32_t)(*reinterpret_cast<const uint16_t*>(P.sites + 2 * cell));
        }
      }
#pragma unroll
      for (int u = 0; u < U; u++) {
        const int ys = ys0 + u;
        if (ys < ey && lane < ex) {
          const int base = hoff(2 * lane, 2 * ys, 2 * zs);
#pragma unroll
          for (int b = 0; b < 4; b++)
            box[base + boff(b)] =
                (uint8_t)(P.storage == SMCX_INT8 ? (v[u] >> (8 * b)) & 0xFFu : (v[u] >> (4 * b)) & 15u);
        }
      }
    }
  }
}
}  // namespace qfcc

// ---------------------------------------------------------------------------
// FCC qSRO sweep with maintained counts.  Every site's same-species counts
// n_k(i) (k < K) live beside its species: in a device array (one 16-bit
// word per site, written by k_qsro_fcc_count_init at the start of each sweep
// call) and, during a tile pass, in a 16-bit shared-memory box (species in
// bits 0..2, n_0 in bits 3..6 (<= 12), n_1 in 7..9 (<= 6), n_2 in 10..14
// (<= 24)).  A trial then reads the count of a changing environment site
// with one load instead of counting its shell, and an accepted swap updates
// the counts it changes: s and s' take the counts the pair loop found, and
// every other environment site i of species a or b that sees s and s' in
// different shells gets its one or two count fields moved by +-1 (one add
// to the packed word; a field never leaves its range, so no carry crosses
// fields).
//
// The box covers the half units [2 t0 - 3, 2 (t0 + ts) + 2] of each axis:
// every site a trial of the tile reads (the two environments) or whose
// count it changes.  Its origin is the odd point 2 t0 - 3, so a site's box
// coordinates have an odd sum, and element (x + y NPX + z NPP + 1) / 2 (odd
// pitches) stores the box's FCC sites without gaps; a lattice vector is a
// constant element offset.  A tile pass writes back the species of the tile
// and its 1-cell ring and the counts of the whole box.  Tiles of one colour
// are at least 3 cells (6 half units) apart, so no two boxes of a launch
// share a site whose count either of them changes or writes.
// ---------------------------------------------------------------------------
namespace qfn {
// Box of tiles of at most TM cells: 2 TM + 6 half units per axis (even), odd
// pitches.  TM = 20 (101 KB, 2 CTAs per SM) and TM = 17 (66 KB, 3 CTAs).
template <int TM>
struct QBox {
  static constexpr int EXT = 2 * TM + 6;
  static constexpr int NPX = EXT + 1;
  static constexpr int NPP = NPX * EXT + 1;
  static constexpr int NELEM = ((EXT - 1) + (EXT - 1) * NPX + (EXT - 1) * NPP + 1) / 2 + 1;
  static constexpr int BOX_BYTES = (NELEM * 2 + 15) / 16 * 16;
  // element of box point (x, y, z), x + y + z odd
  __host__ __device__ static constexpr int eidx(int x, int y, int z) { return (x + y * NPX + z * NPP + 1) / 2; }
  // element offset of a lattice vector (even coordinate sum)
  __host__ __device__ static constexpr int voff(int x, int y, int z) { return (x + y * NPX + z * NPP) / 2; }
};
constexpr int TMAX = 20;
__host__ __device__ constexpr int bx_of(int b) { return (b == 1 || b == 2) ? 1 : 0; }
__host__ __device__ constexpr int by_of(int b) { return (b == 1 || b == 3) ? 1 : 0; }
__host__ __device__ constexpr int bz_of(int b) { return (b == 2 || b == 3) ? 1 : 0; }
__host__ __device__ constexpr int fshift(int k) { return k == 0 ? 3 : k == 1 ? 7 : 10; }
__host__ __device__ constexpr int fmask(int k) { return k == 0 ? 15 : k == 1 ? 7 : 31; }
__device__ __forceinline__ int field_rt(uint32_t v, int k) {
  return k == 0 ? (int)((v >> 3) & 15u) : k == 1 ? (int)((v >> 7) & 7u) : (int)((v >> 10) & 31u);
}
// packed count word of the per-shell counts n[0..K-1]
template <int K>
__device__ __forceinline__ uint32_t pack_counts(const int (&n)[K]) {
  uint32_t w = 0;
#pragma unroll
  for (int k = 0; k < K; k++) w |= (uint32_t)n[k] << (fshift(k) - 3);
  return w;
}
// The environment sites whose counts a trial along partner direction d can
// change, ordered by class so that the kernel's loops see every class at a
// compile-time position: es[d][i] (sites t = s + v of the environment of s,
// class (k1 = shell of t around s, k2 = shell of t around s' or -1 outside
// the K shells), t != s' and k1 != k2), then ep[d][i] (sites t = s' + v
// outside the environment of s and != s, class k = shell around s').  The
// classes' sizes are the same for all 12 directions (they are images of one
// another under the cubic group); `ok` checks that.  Entries are element
// offsets in the count box.
__host__ __device__ constexpr int fcc_shell(int x, int y, int z, int K) {
  const int r = x * x + y * y + z * z;
  const int k = r == 2 ? 0 : r == 4 ? 1 : r == 6 ? 2 : -1;
  return k < K ? k : -1;
}
template <int K>
struct QClass {
  short es[12][42], ep[12][42];
  int k1[42], k2[42], kp[42];  // class of slot i
  int NS, NP;
  bool ok;
};
template <int K, int TM>
__host__ __device__ constexpr QClass<K> make_qclass() {
  constexpr qfcc::QTable T = qfcc::make_qvecs();
  constexpr int NV = vec_count(kFCC, K);
  QClass<K> q{};
  q.ok = true;
  for (int d = 0; d < 12; d++) {
    const int px = T.v[d].x, py = T.v[d].y, pz = T.v[d].z;
    int n = 0;
    for (int a = 0; a < K; a++)
      for (int b = -1; b < K; b++) {
        if (b == a) continue;
        for (int j = 0; j < NV; j++) {
          if (T.v[j].k != a) continue;
          const int ux = T.v[j].x - px, uy = T.v[j].y - py, uz = T.v[j].z - pz;
          if (ux == 0 && uy == 0 && uz == 0) continue;
          if (fcc_shell(ux, uy, uz, K) != b) continue;
          if (d == 0) {
            q.k1[n] = a;
            q.k2[n] = b;
          } else if (q.k1[n] != a || q.k2[n] != b) {
            q.ok = false;
          }
          q.es[d][n++] = (short)QBox<TM>::voff(T.v[j].x, T.v[j].y, T.v[j].z);
        }
      }
    if (d == 0) q.NS = n;
    else if (n != q.NS) q.ok = false;
    int m = 0;
    for (int a = 0; a < K; a++)
      for (int j = 0; j < NV; j++) {
        if (T.v[j].k != a) continue;
        const int wx = T.v[j].x + px, wy = T.v[j].y + py, wz = T.v[j].z + pz;
        if ((wx == 0 && wy == 0 && wz == 0) || fcc_shell(wx, wy, wz, K) >= 0) continue;
        if (d == 0) q.kp[m] = a;
        else if (q.kp[m] != a) q.ok = false;
        q.ep[d][m++] = (short)QBox<TM>::voff(T.v[j].x, T.v[j].y, T.v[j].z);
      }
    if (d == 0) q.NP = m;
    else if (m != q.NP) q.ok = false;
  }
  return q;
}
static_assert(make_qclass<2, 20>().ok && make_qclass<3, 20>().ok, "class sizes differ between partner directions");
__constant__ QClass<2> c_qclass2_20 = make_qclass<2, 20>();
__constant__ QClass<3> c_qclass3_20 = make_qclass<3, 20>();
__constant__ QClass<2> c_qclass2_17 = make_qclass<2, 17>();
__constant__ QClass<3> c_qclass3_17 = make_qclass<3, 17>();
template <int K, int TM>
__device__ __forceinline__ const QClass<K>& qclass() {
  if constexpr (K == 2) return TM == 20 ? c_qclass2_20 : c_qclass2_17;
  else return TM == 20 ? c_qclass3_20 : c_qclass3_17;
}
// Energy change of the environment-of-s slots [I0, I1): a site holding b
// (d = +1) or a (d = -1) sees its count in the shell of s move by d and in
// the shell of s' (if any) by -d; a count n moving by d changes the term by
// W (2 n d + d^2); other species give d = 0.
template <int K, int TM, int I0, int I1>
__device__ __forceinline__ int es_energy(const uint16_t* box, const short* es, int s, int sa, int sb,
                                         const int (&wqa)[K], const int (&wqb)[K]) {
  constexpr QClass<K> QC = make_qclass<K, TM>();
  int dE = 0;
#pragma unroll
  for (int i = I0; i < I1; i++) {
    const uint32_t w = box[s + es[i]];
    const int c = (int)(w & 7u);
    const bool isb = c == sb, isa = c == sa;
    const int d = (int)isb - (int)isa, ad = (int)(isb | isa);
    const int k1 = QC.k1[i], k2 = QC.k2[i];
    const int n1 = (int)((w >> fshift(k1)) & (uint32_t)fmask(k1));
    dE += (isb ? wqb[k1] : wqa[k1]) * (2 * d * n1 + ad);
    if (k2 >= 0) {
      const int n2 = (int)((w >> fshift(k2)) & (uint32_t)fmask(k2));
      dE += (isb ? wqb[k2] : wqa[k2]) * (ad - 2 * d * n2);
    }
  }
  return dE;
}
// The count updates of the same slots after an accepted swap.
template <int K, int TM, int I0, int I1>
__device__ __forceinline__ void es_update(uint16_t* box, const short* es, int s, int sa, int sb) {
  constexpr QClass<K> QC = make_qclass<K, TM>();
#pragma unroll
  for (int i = I0; i < I1; i++) {
    const int t = s + es[i];
    const uint32_t w = box[t];
    const int c = (int)(w & 7u);
    const int d = (int)(c == sb) - (int)(c == sa);
    const int k1 = QC.k1[i], k2 = QC.k2[i];
    const int dw = d * ((1 << fshift(k1)) - (k2 >= 0 ? (1 << fshift(k2)) : 0));
    if (d != 0) box[t] = (uint16_t)((int)w + dw);
  }
}
// Sites around s' outside the environment of s: a site holding a (d = +1)
// or b (d = -1) sees its count in the shell of s' move by d.
template <int K, int TM>
__device__ __forceinline__ int ep_energy(const uint16_t* box, const short* ep, int sp, int sa, int sb,
                                         const int (&wqa)[K], const int (&wqb)[K]) {
  constexpr QClass<K> QC = make_qclass<K, TM>();
  int dE = 0;
#pragma unroll
  for (int i = 0; i < QC.NP; i++) {
    const uint32_t w = box[sp + ep[i]];
    const int c = (int)(w & 7u);
    const bool isb = c == sb, isa = c == sa;
    const int d = (int)isa - (int)isb, ad = (int)(isb | isa);
    const int k = QC.kp[i];
    const int n = (int)((w >> fshift(k)) & (uint32_t)fmask(k));
    dE += (isb ? wqb[k] : wqa[k]) * (2 * d * n + ad);
  }
  return dE;
}
template <int K, int TM>
__device__ __forceinline__ void ep_update(uint16_t* box, const short* ep, int sp, int sa, int sb) {
  constexpr QClass<K> QC = make_qclass<K, TM>();
#pragma unroll
  for (int i = 0; i < QC.NP; i++) {
    const int t = sp + ep[i];
    const uint32_t w = box[t];
    const int c = (int)(w & 7u);
    const int d = (int)(c == sa) - (int)(c == sb);
    if (d != 0) box[t] = (uint16_t)((int)w + d * (1 << fshift(QC.kp[i])));
  }
}
// Pair part around one end: sum_k sum_v W[k][c(e + v)] (SIGN +1 around s,
// -1 around s'), with the counts of species a and b there.
template <int K, int TM, int SIGN>
__device__ __forceinline__ int pair_side(const uint16_t* box, int e, const int32_t* W, int M, int sa, int sb,
                                         int (&na)[K], int (&nb)[K]) {
  constexpr qfcc::QTable T = qfcc::make_qvecs();
  constexpr int NV = vec_count(kFCC, K);
  int dE = 0;
#pragma unroll
  for (int k = 0; k < K; k++) na[k] = nb[k] = 0;
#pragma unroll
  for (int j = 0; j < NV; j++) {
    const int k = T.v[j].k;
    const int c = box[e + QBox<TM>::voff(T.v[j].x, T.v[j].y, T.v[j].z)] & 7;
    dE += SIGN * W[k * M + c];
    na[k] += (c == sa);
    nb[k] += (c == sb);
  }
  return dE;
}
}  // namespace qfn

// Counts of every site of the tile (all tiles in one launch): species staged
// in the even-point box, n_k(i) counted there, one 16-bit
// word per site (n_0 | n_1 << 4 | n_2 << 7) written to cnt[4 cell + b].
template <int K>
__global__ void __launch_bounds__(128) k_qsro_fcc_count_init(const SweepParams P, uint16_t* __restrict__ cnt) {
  using namespace qfcc;
  extern __shared__ __align__(16) unsigned char smem[];
  uint8_t* box = smem;
  int bid = blockIdx.x;
  const int ti[3] = {bid % P.nt[0], (bid / P.nt[0]) % P.nt[1], bid / (P.nt[0] * P.nt[1])};
  int t0[3], ts[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int base = P.n[a] / P.nt[a], rem = P.n[a] % P.nt[a];
    ts[a] = base + (ti[a] < rem ? 1 : 0);
    t0[a] = ti[a] * base + min(ti[a], rem);
  }
  stage_box(P, box, t0, ts);
  __syncthreads();
  const int nx = P.n[0], ny = P.n[1];
  const int ncell = ts[0] * ts[1] * ts[2];
  for (int i = threadIdx.x; i < 4 * ncell; i += blockDim.x) {
    const int b = i & 3, c = i >> 2;
    const int xr = c % ts[0], yr = (c / ts[0]) % ts[1], zr = c / (ts[0] * ts[1]);
    const int t = hoff(2 * (xr + H), 2 * (yr + H), 2 * (zr + H)) + boff(b);
    const int sp = box[t];
    uint32_t w = (uint32_t)count_shell<0>(box, t, sp) | ((uint32_t)count_shell<1>(box, t, sp) << 4);
    if (K > 2) w |= (uint32_t)count_shell<2>(box, t, sp) << 7;
    const long long cell = ((long long)(t0[2] + zr) * ny + (t0[1] + yr)) * nx + (t0[0] + xr);
    cnt[4 * cell + b] = (uint16_t)w;
  }
}

template <int K, int TM>
__global__ void __launch_bounds__(128, TM == 20 ? 2 : 3)
    k_qsro_fcc_n(const SweepParams P, const QsroTables Q, uint16_t* __restrict__ cnt) {
  using namespace qfn;
  using BX = QBox<TM>;
  constexpr int BOX_BYTES = BX::BOX_BYTES;
  constexpr qfcc::QTable T = qfcc::make_qvecs();
  constexpr int NV = vec_count(kFCC, K);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];
  __shared__ int32_t s_wq[kMaxShells * kMaxSweepM];
  constexpr QClass<K> QC = make_qclass<K, TM>();
  constexpr int NS = QC.NS, NP = QC.NP;
  __shared__ short s_es[12 * NS], s_ep[12 * NP];
  __shared__ int s_qoff[NV];

  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  const int M = P.M, KM = K * P.M, MM = P.M * P.M;
  const int nW = MM * KM + MM;
  uint16_t* box = reinterpret_cast<uint16_t*>(smem);
  int32_t* s_w = reinterpret_cast<int32_t*>(smem + BOX_BYTES);

  int bid = blockIdx.x;
  const int jx = bid % P.ntc[0];
  bid /= P.ntc[0];
  const int jy = bid % P.ntc[1];
  const int jz = bid / P.ntc[1];
  const int ti[3] = {2 * jx + (P.tc & 1), 2 * jy + ((P.tc >> 1) & 1), 2 * jz + ((P.tc >> 2) & 1)};
  int t0[3], ts[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int base = P.n[a] / P.nt[a], rem = P.n[a] % P.nt[a];
    ts[a] = base + (ti[a] < rem ? 1 : 0);
    t0[a] = ti[a] * base + min(ti[a], rem);
  }
  if (tid < 3) s_stat[tid] = 0;
  for (int i = tid; i < nW; i += nth) s_w[i] = P.wtab[i];
  for (int i = tid; i < KM; i += nth) s_wq[i] = Q.W[i];
  for (int i = tid; i < 12 * NS; i += nth) s_es[i] = (qclass<K, TM>().es)[i / NS][i % NS];
  for (int i = tid; i < 12 * NP; i += nth) s_ep[i] = (qclass<K, TM>().ep)[i / NP][i % NP];
  if (tid < NV) {
    int o = 0;
#pragma unroll
    for (int j = 0; j < NV; j++)
      if (j == tid) o = BX::voff(T.v[j].x, T.v[j].y, T.v[j].z);
    s_qoff[tid] = o;  // the first 12 entries are the partner offsets
  }

  // stage the cells [t0 - 2, t0 + ts + 2) of each axis: species and counts,
  // the sites inside the box (box coordinate 2 i - 1 + basis in [0, 2 ts + 5])
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const int ex = ts[0] + 4, ey = ts[1] + 4, ez = ts[2] + 4;
  const int lim[3] = {2 * ts[0] + 5, 2 * ts[1] + 5, 2 * ts[2] + 5};
  {
    // one box column per lane (ex <= 24 < 32), warp w the planes w, w +
    // nwarp, ..., the loads of U rows of a plane issued before any is
    // unpacked
    constexpr int U = 8;
    const int gx = lane < ex ? wrap_add(t0[0] - 2, lane, nx) : 0;
    for (int zs = warp; zs < ez; zs += nwarp) {
      const long long zrow = (long long)wrap_add(t0[2] - 2, zs, nz) * ny;
      for (int ys0 = 0; ys0 < ey; ys0 += U) {
        uint32_t v[U];
        uint2 c4[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          v[u] = 0;
          c4[u] = make_uint2(0, 0);
          if (ys < ey && lane < ex) {
            const long long cell = (zrow + wrap_add(t0[1] - 2, ys, ny)) * nx + gx;
            v[u] = P.storage == SMCX_INT8 ? *reinterpret_cast<const uint32_t*>(P.sites + 4 * cell)
                                          : (uint32_t)(*reinterpret_cast<const uint16_t*>(P.sites + 2 * cell));
            c4[u] = *reinterpret_cast<const uint2*>(cnt + 4 * cell);
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
          const int ys = ys0 + u;
          if (ys < ey && lane < ex) {
#pragma unroll
            for (int b = 0; b < 4; b++) {
              const int x = 2 * lane - 1 + bx_of(b), y = 2 * ys - 1 + by_of(b), z = 2 * zs - 1 + bz_of(b);
              if (x < 0 || y < 0 || z < 0 || x > lim[0] || y > lim[1] || z > lim[2]) continue;
              const uint32_t sp = P.storage == SMCX_INT8 ? (v[u] >> (8 * b)) & 0xFFu : (v[u] >> (4 * b)) & 15u;
              const uint32_t cw = ((b < 2 ? c4[u].x : c4[u].y) >> (16 * (b & 1))) & 0xFFFFu;
              box[BX::eidx(x, y, z)] = (uint16_t)(sp | (cw << 3));
            }
          }
        }
      }
    }
  }
  __syncthreads();

  unsigned long long acc = 0, same = 0;
  long long dsum = 0;
  const int L = P.L;
  const int NQ = (max(ts[0], max(ts[1], ts[2])) + L - 1) / L;
  const int qx = tid % NQ, qy = (tid / NQ) % NQ, qz = tid / (NQ * NQ);
  const bool slot = tid < NQ * NQ * NQ;
  for (int cz = 0; cz < L; cz++)
    for (int cy = 0; cy < L; cy++)
      for (int cx = 0; cx < L; cx++) {
        const int xr = cx + L * qx, yr = cy + L * qy, zr = cz + L * qz;
        const bool here = slot && xr < ts[0] && yr < ts[1] && zr < ts[2];
        const int cbase = BX::eidx(2 * xr + 3, 2 * yr + 3, 2 * zr + 3);
        const unsigned long long cell = ((unsigned long long)(t0[2] + zr) * ny + (t0[1] + yr)) * nx + (t0[0] + xr);
        uint4 rw = make_uint4(0, 0, 0, 0);
        for (int b = 0; b < 4; b++) {
          if (here) {
            if ((b & 1) == 0) rw = attempt_block(cell * 4 + b, P.sweep, P.replica, P.seed_lo, P.seed_hi);
            const uint32_t rd = (b & 1) ? rw.z : rw.x;
            const uint32_t ru = (b & 1) ? rw.w : rw.y;
            const int s = cbase + BX::voff(bx_of(b), by_of(b), bz_of(b));
            const int dir = (int)__umulhi(rd, 12u);
            const int sp = s + s_qoff[dir];
            const int sa = box[s] & 7, sb = box[sp] & 7;
            if (sa == sb) {
              same++;
            } else {
              const int32_t* W = s_w + (sa * M + sb) * KM;
              int wqa[K], wqb[K];
#pragma unroll
              for (int k = 0; k < K; k++) {
                wqa[k] = s_wq[k * M + sa];
                wqb[k] = s_wq[k * M + sb];
              }
              // pair part and the counts of s and s' after the swap: b
              // around s without s' (which holds b before the swap), a around
              // s' without s
              int na_s[K], nb_s[K], na_p[K], nb_p[K];
              int dE = s_w[MM * KM + sa * M + sb] + pair_side<K, TM, 1>(box, s, W, M, sa, sb, na_s, nb_s) +
                       pair_side<K, TM, -1>(box, sp, W, M, sa, sb, na_p, nb_p);
              nb_s[0]--;
              na_p[0]--;
#pragma unroll
              for (int k = 0; k < K; k++)
                dE += wqb[k] * (nb_s[k] * nb_s[k] - nb_p[k] * nb_p[k]) + wqa[k] * (na_p[k] * na_p[k] - na_s[k] * na_s[k]);
              // environment sites whose counts move
              const short* es = s_es + dir * NS;
              const short* ep = s_ep + dir * NP;
              dE += es_energy<K, TM, 0, NS>(box, es, s, sa, sb, wqa, wqb);
              dE += ep_energy<K, TM>(box, ep, sp, sa, sb, wqa, wqb);
              if (metropolis_accept(dE, ru, P.thr, P.nA, P.thr + kNA)) {
                box[s] = (uint16_t)(sb | (pack_counts<K>(nb_s) << 3));
                box[sp] = (uint16_t)(sa | (pack_counts<K>(na_p) << 3));
                es_update<K, TM, 0, NS>(box, es, s, sa, sb);
                ep_update<K, TM>(box, ep, sp, sa, sb);
                acc++;
                dsum += dE;
              }
            }
          }
          __syncthreads();
        }
      }

  // write back the species of the tile and its 1-cell ring, the counts of
  // every site in the box
  const int gxs = lane < ex ? wrap_add(t0[0] - 2, lane, nx) : 0;
  for (int zs = warp; zs < ez; zs += nwarp) {
    const long long zrow = (long long)wrap_add(t0[2] - 2, zs, nz) * ny;
#pragma unroll 2
    for (int ys = 0; ys < ey; ys++) {
      if (lane < ex) {
        const int xs = lane;
        const long long cell = (zrow + wrap_add(t0[1] - 2, ys, ny)) * nx + gxs;
        uint32_t w4[4];
        bool in[4];
#pragma unroll
        for (int b = 0; b < 4; b++) {
          const int x = 2 * xs - 1 + bx_of(b), y = 2 * ys - 1 + by_of(b), z = 2 * zs - 1 + bz_of(b);
          in[b] = !(x < 0 || y < 0 || z < 0 || x > lim[0] || y > lim[1] || z > lim[2]);
          w4[b] = in[b] ? box[BX::eidx(x, y, z)] : 0u;
        }
        if (in[0] && in[1] && in[2] && in[3]) {
          *reinterpret_cast<uint2*>(cnt + 4 * cell) =
              make_uint2((w4[0] >> 3) | ((w4[1] >> 3) << 16), (w4[2] >> 3) | ((w4[3] >> 3) << 16));
        } else {
#pragma unroll
          for (int b = 0; b < 4; b++)
            if (in[b]) cnt[4 * cell + b] = (uint16_t)(w4[b] >> 3);
        }
        const bool ring = xs >= 1 && xs <= ts[0] + 2 && ys >= 1 && ys <= ts[1] + 2 && zs >= 1 && zs <= ts[2] + 2;
        if (ring) {
          if (P.storage == SMCX_INT8)
            *reinterpret_cast<uint32_t*>(P.sites + 4 * cell) =
                (w4[0] & 7u) | ((w4[1] & 7u) << 8) | ((w4[2] & 7u) << 16) | ((w4[3] & 7u) << 24);
          else
            *reinterpret_cast<uint16_t*>(P.sites + 2 * cell) =
                (uint16_t)((w4[0] & 7u) | ((w4[1] & 7u) << 4) | ((w4[2] & 7u) << 8) | ((w4[3] & 7u) << 12));
        }
      }
    }
  }
  add_stats_warp(s_stat, (unsigned)acc, (unsigned)same, dsum);
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&P.stats[0], (unsigned long long)ts[0] * ts[1] * ts[2] * 4);
    atomicAdd(&P.stats[1], s_stat[0]);
    atomicAdd(&P.stats[2], s_stat[1]);
    atomicAdd(&P.stats[3], s_stat[2]);
  }
}

// sum_i sum_k W[k][s_i] n_k(i)^2 added to *E (global-memory gathers).
template <int KIND, int K>
__global__ void __launch_bounds__(256) k_qsro_energy(const SweepParams P, const QsroTables Q, long long* E) {
  constexpr int m = cell_sites(KIND);
  __shared__ long long part[8];
  __shared__ int32_t s_wq[kMaxShells * kMaxSweepM];
  for (int i = threadIdx.x; i < K * P.M; i += blockDim.x) s_wq[i] = Q.W[i];
  __syncthreads();
  const long long ncell = (long long)P.n[0] * P.n[1] * P.n[2];
  long long acc = 0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % P.n[0]);
    const long long r = c / P.n[0];
    const int y = (int)(r % P.n[1]), z = (int)(r / P.n[1]);
    for (int b = 0; b < m; b++) {
      const int p = load_site(P.sites, c * m + b, P.storage);
      int j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
        int n = 0;
        for (int q = 0; q < shell_size(KIND, k); q++, j++) {
          const signed char* d = P.gd[b][j];
          const long long t =
              (((long long)wrap_add(z, d[2], P.n[2]) * P.n[1] + wrap_add(y, d[1], P.n[1])) * P.n[0] +
               wrap_add(x, d[0], P.n[0])) * m + d[3];
          n += (load_site(P.sites, t, P.storage) == p);
        }
        acc += (long long)s_wq[k * P.M + p] * n * n;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) t += part[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(E), (unsigned long long)t);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

void fill_offsets_global(const smcx_lattice* hd, SweepParams& P);

namespace {

int shell_index(const Shells& S, int x, int y, int z) {
  for (int j = 0; j < S.nv; j++)
    if (S.v[j][0] == x && S.v[j][1] == y && S.v[j][2] == z) return S.shell_of[j];
  return -1;
}

QsroTables make_tables(const smcx_lattice* hd) {
  QsroTables T;
  memset(&T, 0, sizeof(T));
  const Shells& S = hd->shells;
  for (size_t i = 0; i < hd->Wq.size(); i++) T.W[i] = hd->Wq[i];
  for (int d = 0; d < S.z[0]; d++)
    for (int j = 0; j < S.nv; j++) {
      const int* p = S.v[d];
      const int* v = S.v[j];
      const int ux = p[0] - v[0], uy = p[1] - v[1], uz = p[2] - v[2];
      T.k2[d][j] = (ux == 0 && uy == 0 && uz == 0) ? -2 : (signed char)shell_index(S, ux, uy, uz);
      const int wx = p[0] + v[0], wy = p[1] + v[1], wz = p[2] + v[2];
      T.in_s[d][j] = ((wx == 0 && wy == 0 && wz == 0) || shell_index(S, wx, wy, wz) >= 0) ? 1 : 0;
    }
  for (int b = 0; b < hd->m; b++) {
    int B[3];
    basis_of(hd->kind, b, B);
    for (int j = 0; j < S.nv; j++) {
      int r[3];
      for (int a = 0; a < 3; a++) {
        const int q = B[a] + S.v[j][a];
        const int d = (q >= 0) ? q / 2 : -((-q + 1) / 2);
        r[a] = q - 2 * d;
      }
      T.sub[b][j] = (signed char)basis_index(hd->kind, r[0], r[1], r[2]);
    }
  }
  int o = 0;
  for (int k = 0; k < S.K; k++) {
    T.start[k] = (unsigned char)o;
    o += S.z[k];
  }
  T.start[S.K] = (unsigned char)o;
  return T;
}

void fill_tile_offsets(const smcx_lattice* hd, SweepParams& P) {
  const Shells& S = hd->shells;
  const int m = hd->m;
  for (int b = 0; b < m; b++) {
    int B[3];
    basis_of(hd->kind, b, B);
    for (int j = 0; j < S.nv; j++) {
      int d[3], r[3];
      for (int a = 0; a < 3; a++) {
        const int q = B[a] + S.v[j][a];
        d[a] = (q >= 0) ? q / 2 : -((-q + 1) / 2);
        r[a] = q - 2 * d[a];
      }
      const int bb = basis_index(hd->kind, r[0], r[1], r[2]);
      P.off[b][j] = ((d[2] * P.BY + d[1]) * P.BX + d[0]) * m + (bb - b);
      if (j < S.z[0]) {
        P.poff[b][j] = P.off[b][j];
        P.psub[b][j] = bb;
      }
    }
  }
}

template <int KIND, int K>
void launch_qsro(smcx_lattice* hd, SweepParams& P, const QsroTables& T, int64_t n_sweeps, int n_colours) {
  constexpr int m = cell_sites(KIND);
  constexpr int NV = vec_count(KIND, K);
  constexpr int Z1 = shell_size(KIND, 0);
  const int nW = P.M * P.M * K * P.M + P.M * P.M;
  const size_t smem = (size_t)(nW + P.nA + kNB + m * NV + 2 * m * Z1) * 4 + (size_t)P.BX * P.BY * P.BZ * m;
  if (smem > 200 * 1024) fail(SMCX_E_UNSUPPORTED, "tile too large for shared memory");
  int slots = 1;
  for (int a = 0; a < 3; a++) slots *= ((P.n[a] + P.nt[a] - 1) / P.nt[a] + P.L - 1) / P.L;
  auto run = [&](auto kern, int nt) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "qSRO sweep smem attribute");
    for (int64_t s = 0; s < n_sweeps; s++) {
      P.sweep = hd->sweep_cum + (uint64_t)s;
      for (int tc = 0; tc < n_colours; tc++) {
        P.tc = tc;
        const int grid = P.ntc[0] * P.ntc[1] * P.ntc[2];
        kern<<<grid, nt, smem, hd->stream>>>(P, T);
      }
    }
  };
  if (slots <= 128) run(k_tile_sweep_qsro<KIND, K, 128>, 128);
  else run(k_tile_sweep_qsro<KIND, K, 256>, 256);
  check_cuda(cudaGetLastError(), "qSRO sweep launch");
}

}  // namespace

void sweep_qsro_device(smcx_lattice* hd, int nA, uint64_t seed, int64_t n_sweeps, int n_colours) {
  const smcx_sched& sc = hd->sched;
  if (hd->proposal != SMCX_PROPOSAL_SITE) fail(SMCX_E_UNSUPPORTED, "qSRO sweeps use per-trial directions");
  for (int a = 0; a < 3; a++)
    if (sc.nt[a] < 2) fail(SMCX_E_UNSUPPORTED, "qSRO sweeps run tiled schedules (>= 2 tiles per axis)");
  SweepParams P;
  memset(&P, 0, sizeof(P));
  P.sites = hd->d_sites;
  P.thr = hd->d_thr;
  P.wtab = hd->d_wtab;
  P.stats = hd->d_stats;
  for (int a = 0; a < 3; a++) {
    P.n[a] = hd->n[a];
    P.nt[a] = sc.nt[a];
    P.ntc[a] = sc.nt[a] / 2;
  }
  P.L = sc.L;
  P.h = halo_cells(hd->shells);
  P.ring = ring_cells(hd->shells);
  int tmax[3];
  for (int a = 0; a < 3; a++) tmax[a] = (hd->n[a] + sc.nt[a] - 1) / sc.nt[a];
  P.BX = tmax[0] + 2 * P.h;
  P.BY = tmax[1] + 2 * P.h;
  P.BZ = tmax[2] + 2 * P.h;
  P.M = hd->M;
  P.nA = nA;
  P.storage = hd->storage;
  P.replica = hd->replica;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  fill_tile_offsets(hd, P);
  const QsroTables T = make_tables(hd);
  const int K = hd->shells.K;
  // FCC with tiles of at most 20 cells, link cells >= 4, 5^3 slots at most,
  // a 4-byte aligned store: the even-point kernel
  const int tm = std::max(tmax[0], std::max(tmax[1], tmax[2]));
  const int tmin = std::min(hd->n[0] / sc.nt[0], std::min(hd->n[1] / sc.nt[1], hd->n[2] / sc.nt[2]));
  const int nq = (tm + sc.L - 1) / sc.L;
  // FCC, 2 or 3 shells, tiles of 3 to 20 cells: the maintained-count kernel,
  // after one launch that counts every site's same-species neighbours (tiles
  // of >= 3 cells keep the boxes of one colour, and a box and its own
  // periodic image, apart)
  if (hd->kind == kFCC && (K == 2 || K == 3) && tm <= qfn::TMAX && tmin >= 3 && nq * nq * nq <= 128 &&
      reinterpret_cast<uintptr_t>(P.sites) % 4 == 0) {
    const long long ncell = (long long)hd->n[0] * hd->n[1] * hd->n[2];
    if (!hd->d_qcnt) check_cuda(cudaMalloc(&hd->d_qcnt, (size_t)ncell * 4 * sizeof(uint16_t)), "qSRO count array");
    auto init = K == 2 ? k_qsro_fcc_count_init<2> : k_qsro_fcc_count_init<3>;
    check_cuda(cudaFuncSetAttribute(init, cudaFuncAttributeMaxDynamicSharedMemorySize, qfcc::BOX_BYTES),
               "qSRO count smem attribute");
    init<<<sc.nt[0] * sc.nt[1] * sc.nt[2], 128, qfcc::BOX_BYTES, hd->stream>>>(P, hd->d_qcnt);
    const int nW = P.M * P.M * K * P.M + P.M * P.M;
    const bool small = tm <= 17;  // the 66 KB box: three CTAs per SM
    const size_t smem = (small ? qfn::QBox<17>::BOX_BYTES : qfn::QBox<20>::BOX_BYTES) + (size_t)nW * 4;
    auto kern = K == 2 ? (small ? k_qsro_fcc_n<2, 17> : k_qsro_fcc_n<2, 20>)
                       : (small ? k_qsro_fcc_n<3, 17> : k_qsro_fcc_n<3, 20>);
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "qSRO FCC smem attribute");
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100), "qSRO FCC carveout");
    for (int64_t sw = 0; sw < n_sweeps; sw++) {
      P.sweep = hd->sweep_cum + (uint64_t)sw;
      for (int tc = 0; tc < n_colours; tc++) {
        P.tc = tc;
        kern<<<P.ntc[0] * P.ntc[1] * P.ntc[2], 128, smem, hd->stream>>>(P, T, hd->d_qcnt);
      }
    }
    check_cuda(cudaGetLastError(), "qSRO FCC sweep launch");
    return;
  }
  if (hd->kind == kBCC) {
    switch (K) {
      case 1: launch_qsro<kBCC, 1>(hd, P, T, n_sweeps, n_colours); break;
      case 2: launch_qsro<kBCC, 2>(hd, P, T, n_sweeps, n_colours); break;
      case 3: launch_qsro<kBCC, 3>(hd, P, T, n_sweeps, n_colours); break;
      default: launch_qsro<kBCC, 4>(hd, P, T, n_sweeps, n_colours); break;
    }
  } else {
    switch (K) {
      case 1: launch_qsro<kFCC, 1>(hd, P, T, n_sweeps, n_colours); break;
      case 2: launch_qsro<kFCC, 2>(hd, P, T, n_sweeps, n_colours); break;
      default: launch_qsro<kFCC, 3>(hd, P, T, n_sweeps, n_colours); break;
    }
  }
}

void qsro_energy_add(smcx_lattice* hd) {
  SweepParams P;
  memset(&P, 0, sizeof(P));
  P.sites = hd->d_sites;
  P.M = hd->M;
  P.storage = hd->storage;
  for (int a = 0; a < 3; a++) P.n[a] = hd->n[a];
  fill_offsets_global(hd, P);
  const QsroTables T = make_tables(hd);
  int dev = 0, nsm = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "SM count");
  const long long ncell = (long long)hd->n[0] * hd->n[1] * hd->n[2];
  const int grid = (int)std::max<long long>(1, std::min<long long>((ncell + 255) / 256, (long long)nsm * 8));
  const int K = hd->shells.K;
  auto go = [&](auto kern) { kern<<<grid, 256, 0, hd->stream>>>(P, T, hd->d_energy); };
  if (hd->kind == kBCC) {
    switch (K) {
      case 1: go(k_qsro_energy<kBCC, 1>); break;
      case 2: go(k_qsro_energy<kBCC, 2>); break;
      case 3: go(k_qsro_energy<kBCC, 3>); break;
      default: go(k_qsro_energy<kBCC, 4>); break;
    }
  } else {
    switch (K) {
      case 1: go(k_qsro_energy<kFCC, 1>); break;
      case 2: go(k_qsro_energy<kFCC, 2>); break;
      default: go(k_qsro_energy<kFCC, 3>); break;
    }
  }
  check_cuda(cudaGetLastError(), "qSRO energy launch");
}

}  // namespace smcx
