// Ordered pair counts of a BCC lattice (M <= 4) from shared-memory tiles.
//
// Same result as k_pair_counts (smcx_aux.cu): C[k][p][q] = number of (site
// i, shell-k vector v) with s_i = p and s_{i+v} = q.  Every unordered pair is
// visited once: with H_k the half of shell k whose first nonzero component is
// positive, U[k][p][q] = #(i, v in H_k) with s_i = p, s_{i+v} = q, and on a
// periodic lattice the vector -v contributes U[k][q][p] (substitute i -> i+v
// in the sum), so C[k][p][q] = U[k][p][q] + U[k][q][p].
// Each CTA stages one tile plus its 2-cell halo exactly as the sweep does,
// and for every site of the tile adds 1 << (8 s_{i+v}) over the half-shell
// vectors into a byte-packed register, which is split into two 16-bit-field
// accumulators per (shell, centre species).  At the end the warp sums each
// accumulator with a reduce-add, lane 0 adds the unpacked counts to a shared
// histogram U, and the CTA adds U and its transpose to the global int64
// histogram.
#include "smcx_bcc_tile.cuh"

namespace smcx {

namespace bccfast {

// The tile of this CTA (tiles numbered x fastest) and its staging: tile plus
// a 2-cell halo into the sublattice byte arrays of the sweep's box layout,
// species stored as 8 s.
__device__ __forceinline__ void tile_of_index(const LatDesc& D, int t, int t0[3], int ts[3]) {
  const int ntx = D.nt[0], nty = D.nt[1];
  const int ti[3] = {t % ntx, (t / ntx) % nty, t / (ntx * nty)};
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const int base = D.n[a] / D.nt[a], rem = D.n[a] % D.nt[a];
    ts[a] = base + (ti[a] < rem ? 1 : 0);
    t0[a] = ti[a] * base + min(ti[a], rem);
  }
}

__device__ __forceinline__ void stage_tile(const LatDesc& D, uint8_t* box, const int t0[3], const int ts[3]) {
  stage_box(D, box, t0, ts, threadIdx.x & 31, threadIdx.x >> 5, blockDim.x >> 5);
}

// Exact division of 0 <= c < 2^16 by 2 <= d < 2^10 with a 32-bit multiply-high
// by m = ceil(2^32 / d): c m / 2^32 = c / d + c e / 2^32 with 0 <= e < 1, and
// c e / 2^32 < 2^-16 < 1 / d, so the floor is c / d (d = 1 passes c through).
struct FastDiv {
  uint32_t d, m;
  __device__ __forceinline__ explicit FastDiv(uint32_t dd)
      : d(dd), m(dd > 1 ? (uint32_t)((0xFFFFFFFFull) / dd + 1) : 0u) {}
  __device__ __forceinline__ uint32_t div(uint32_t c) const { return d > 1 ? __umulhi(c, m) : c; }
};

// Cell c of a tile of ts[0] x ts[1] x ts[2] cells (x fastest).
struct CellIndex {
  FastDiv dx, dxy;
  __device__ __forceinline__ CellIndex(const int ts[3]) : dx((uint32_t)ts[0]), dxy((uint32_t)(ts[0] * ts[1])) {}
  __device__ __forceinline__ void at(int c, int& xr, int& yr, int& zr) const {
    const uint32_t z = dxy.div((uint32_t)c);
    const uint32_t r = (uint32_t)c - z * dxy.d;
    const uint32_t y = dx.div(r);
    zr = (int)z;
    yr = (int)y;
    xr = (int)(r - y * dx.d);
  }
};

// Half of a shell: the vectors whose first nonzero half-unit component is
// positive (one of each +v / -v pair).
__host__ __device__ constexpr bool half_vec(const Vec& v) {
  return v.x > 0 || (v.x == 0 && (v.y > 0 || (v.y == 0 && v.z > 0)));
}

// Pair counts of tile t of lattice D added into counts [K][M][M].
template <int K>
__device__ __forceinline__ void pair_counts_tile(const LatDesc& D, int t, unsigned long long* __restrict__ counts,
                                                 uint8_t* box, unsigned int* hist) {
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31;
  int t0[3], ts[3];
  tile_of_index(D, t, t0, ts);
  for (int i = tid; i < kMaxShells * 16; i += nth) hist[i] = 0;
  constexpr int h = 2;
  stage_tile(D, box, t0, ts);
  __syncthreads();

  // acc[k][p][0] holds bytes 0 and 2 of the per-site counters, acc[k][p][1]
  // bytes 1 and 3, each in a 16-bit field (no overflow below 2700 sites)
  uint32_t acc[K][4][2];
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int p = 0; p < 4; p++) acc[k][p][0] = acc[k][p][1] = 0;
  const int ncell = ts[0] * ts[1] * ts[2];
  constexpr VecTable T = make_vecs();
  const CellIndex ci(ts);
  for (int c = tid; c < ncell; c += nth) {
    int xr, yr, zr;
    ci.at(c, xr, yr, zr);
    const int s0 = (zr + h) * PP + (yr + h) * PX + (xr + h);
#pragma unroll
    for (int B = 0; B < 2; B++) {
      const int s = s0 + B * SUB;
      const int p = box[s] >> 3;
      uint32_t hk[K];
#pragma unroll
      for (int k = 0; k < K; k++) hk[k] = 0;
#pragma unroll
      for (int j = 0; j < T.n; j++) {
        const int k = T.v[j].k;
        if (k >= K) continue;
        if (!half_vec(T.v[j])) continue;
        const int off = B == 0 ? nb_offset(0, T.v[j].x, T.v[j].y, T.v[j].z) : nb_offset(1, T.v[j].x, T.v[j].y, T.v[j].z);
        hk[k] += 1u << box[s + off];
      }
#pragma unroll
      for (int k = 0; k < K; k++) {
        const uint32_t lo = hk[k] & 0x00FF00FFu, hi = (hk[k] >> 8) & 0x00FF00FFu;
#pragma unroll
        for (int pp = 0; pp < 4; pp++)
          if (p == pp) {
            acc[k][pp][0] += lo;
            acc[k][pp][1] += hi;
          }
      }
    }
  }
  // warp sums (16-bit fields: at most 32 lanes x 32 cells x 2 sites x 12 = 24576 per field)
#pragma unroll
  for (int k = 0; k < K; k++)
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
      for (int w = 0; w < 2; w++) {
        const uint32_t v = __reduce_add_sync(0xffffffffu, acc[k][p][w]);
        if (lane == 0) {
          // field 0 -> species q = w, field 1 -> species q = w + 2
          atomicAdd(&hist[(k * 4 + p) * 4 + w], v & 0xFFFFu);
          atomicAdd(&hist[(k * 4 + p) * 4 + w + 2], v >> 16);
        }
      }
  __syncthreads();
  for (int i = tid; i < K * 16; i += nth) {
    const int k = i / 16, p = (i / 4) % 4, q = i % 4;
    if (p < D.M && q < D.M && hist[i]) {
      atomicAdd(&counts[(k * D.M + p) * D.M + q], (unsigned long long)hist[i]);
      atomicAdd(&counts[(k * D.M + q) * D.M + p], (unsigned long long)hist[i]);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_bcc_pair_counts(const LatDesc D, unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int hist[kMaxShells * 16];
  pair_counts_tile<K>(D, blockIdx.x, counts, smem, hist);
}

// Many lattices in one launch: CTA i takes tile items[i].y of lattice
// items[i].x and adds into counts + items[i].x * kmm.
template <int K>
__global__ void __launch_bounds__(256) k_bcc_pair_counts_multi(const LatDesc* __restrict__ descs,
                                                              const int2* __restrict__ items, int kmm,
                                                              unsigned long long* __restrict__ counts) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned int hist[kMaxShells * 16];
  const int2 it = items[blockIdx.x];
  const LatDesc D = descs[it.x];
  pair_counts_tile<K>(D, it.y, counts + (size_t)it.x * kmm, smem, hist);
}

// Energy directly (M <= 4): E = sum_i sum_k sum_{v in half shell k}
// V_k[s_i][s_{i+v}], every unordered pair once.  Per site the half-shell
// neighbours go into byte-packed per-species counters h_k (at most 12 per
// byte), and the site's term is sum_k dp4a(h_k, row of V_k for its species)
// over the byte planes of V (two or three planes, |V| < 2^23), the rows read
// from a shared table indexed by the site's species.
template <int K, int PL>
__global__ void __launch_bounds__(256) k_bcc_energy(const LatDesc D, const Planes Q, long long* __restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t sP[PL * kMaxShells * 4];
  __shared__ long long part[8];
  uint8_t* box = smem;
  const int tid = threadIdx.x, nth = blockDim.x;
  int t0[3], ts[3];
  tile_of_index(D, blockIdx.x, t0, ts);
  for (int i = tid; i < PL * K * 4; i += nth) sP[i] = Q.P[i / (K * 4)][(i / 4) % K][i % 4][0];
  constexpr int h = 2;
  stage_tile(D, box, t0, ts);
  __syncthreads();
  long long acc = 0;
  const int ncell = ts[0] * ts[1] * ts[2];
  constexpr VecTable T = make_vecs();
  const CellIndex ci(ts);
  for (int c = tid; c < ncell; c += nth) {
    int xr, yr, zr;
    ci.at(c, xr, yr, zr);
    const int s0 = (zr + h) * PP + (yr + h) * PX + (xr + h);
    int g = 0;
#pragma unroll
    for (int B = 0; B < 2; B++) {
      const int s = s0 + B * SUB;
      const int p = box[s] >> 3;
      uint32_t hk[K];
#pragma unroll
      for (int k = 0; k < K; k++) hk[k] = 0;
#pragma unroll
      for (int j = 0; j < T.n; j++) {
        const int k = T.v[j].k;
        if (k >= K || !half_vec(T.v[j])) continue;
        const int off = B == 0 ? nb_offset(0, T.v[j].x, T.v[j].y, T.v[j].z) : nb_offset(1, T.v[j].x, T.v[j].y, T.v[j].z);
        hk[k] += 1u << box[s + off];
      }
      int a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
        a0 = dp4a_su((int)hk[k], sP[(0 * K + k) * 4 + p], a0);
        if (PL == 2) {
          a1 = dp4a_ss((int)hk[k], sP[(1 * K + k) * 4 + p], a1);
        } else {
          a1 = dp4a_su((int)hk[k], sP[(1 * K + k) * 4 + p], a1);
          a2 = dp4a_ss((int)hk[k], sP[(2 * K + k) * 4 + p], a2);
        }
      }
      g += a0 + (a1 << 8) + (a2 << 16);
    }
    acc += g;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) part[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    long long t = 0;
    for (int w = 0; w < nth / 32; w++) t += part[w];
    atomicAdd(reinterpret_cast<unsigned long long*>(E), (unsigned long long)t);
  }
}

}  // namespace bccfast

// Usable for BCC, M <= 4, tiles (of the handle's schedule, or a default
// tiling) that fit the 24^3 box.
bool bcc_counts_usable(const smcx_lattice* hd, int nt[3]) {
  if (hd->kind != kBCC || hd->M > 4 || !hd->have_epi) return false;
  const smcx_sched& sc = hd->sched;
  for (int a = 0; a < 3; a++) {
    int t = (sc.L != 0 && sc.nt[a] >= 2) ? sc.nt[a] : std::max(1, (hd->n[a] + 19) / 20);
    while ((hd->n[a] + t - 1) / t > 20) t++;
    if (hd->n[a] / t < 1) return false;
    nt[a] = t;
    if ((hd->n[a] + t - 1) / t + 4 > bccfast::BOX) return false;
  }
  // a tile covering a whole axis would wrap its own halo: the generic kernel
  // handles those small lattices
  for (int a = 0; a < 3; a++)
    if (nt[a] < 2 || hd->n[a] < 6) return false;
  return true;
}

void pair_counts_bcc_tiled(smcx_lattice* hd, const int nt[3]) {
  bccfast::LatDesc D;
  memset(&D, 0, sizeof(D));
  D.sites = hd->d_sites;
  D.storage = hd->storage;
  D.M = hd->M;
  for (int a = 0; a < 3; a++) {
    D.n[a] = hd->n[a];
    D.nt[a] = nt[a];
  }
  const int grid = nt[0] * nt[1] * nt[2];
  const size_t smem = 2 * bccfast::SUB;
  auto go = [&](auto kern) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
    kern<<<grid, 256, smem, hd->stream>>>(D, hd->d_counts);
  };
  switch (hd->shells.K) {
    case 1: go(bccfast::k_bcc_pair_counts<1>); break;
    case 2: go(bccfast::k_bcc_pair_counts<2>); break;
    case 3: go(bccfast::k_bcc_pair_counts<3>); break;
    default: go(bccfast::k_bcc_pair_counts<4>); break;
  }
  check_cuda(cudaGetLastError(), "tiled pair-count launch");
}

int build_planes(const smcx_lattice* hd, bccfast::Planes* Q, int min_planes);

// Pair counts of many BCC lattices (M <= 4, K shells) in one launch: d_descs
// [R] and d_items [n_items] (lattice, tile) on the device, counts [R][K][M][M]
// zeroed by the caller.
void pair_counts_bcc_multi(const bccfast::LatDesc* d_descs, const int2* d_items, int n_items, int K, int M,
                           unsigned long long* d_counts, cudaStream_t st) {
  const size_t smem = 2 * bccfast::SUB;
  const int kmm = K * M * M;
  auto go = [&](auto kern) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
    kern<<<n_items, 256, smem, st>>>(d_descs, d_items, kmm, d_counts);
  };
  switch (K) {
    case 1: go(bccfast::k_bcc_pair_counts_multi<1>); break;
    case 2: go(bccfast::k_bcc_pair_counts_multi<2>); break;
    case 3: go(bccfast::k_bcc_pair_counts_multi<3>); break;
    default: go(bccfast::k_bcc_pair_counts_multi<4>); break;
  }
  check_cuda(cudaGetLastError(), "batched pair-count launch");
}

// Energy of a BCC lattice with M <= 4 straight from the tiles (no pair-count
// histogram); false when the tiled path does not apply.
bool energy_bcc_direct(smcx_lattice* hd) {
  int nt[3];
  if (hd->kernel_choice == SMCX_KERNEL_GENERIC || !bcc_counts_usable(hd, nt)) return false;
  for (int32_t v : hd->V)
    if (v >= (1 << 23) || v <= -(1 << 23)) return false;
  bccfast::LatDesc D;
  memset(&D, 0, sizeof(D));
  D.sites = hd->d_sites;
  D.storage = hd->storage;
  D.M = hd->M;
  for (int a = 0; a < 3; a++) {
    D.n[a] = hd->n[a];
    D.nt[a] = nt[a];
  }
  bccfast::Planes Q;
  const int PL = build_planes(hd, &Q, 2);
  const int grid = nt[0] * nt[1] * nt[2];
  const size_t smem = 2 * bccfast::SUB;
  check_cuda(cudaMemsetAsync(hd->d_energy, 0, sizeof(long long), hd->stream), "clear energy");
  auto go = [&](auto kern) {
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "smem attr");
    kern<<<grid, 256, smem, hd->stream>>>(D, Q, hd->d_energy);
  };
  const int K = hd->shells.K;
  if (PL == 2) {
    switch (K) {
      case 1: go(bccfast::k_bcc_energy<1, 2>); break;
      case 2: go(bccfast::k_bcc_energy<2, 2>); break;
      case 3: go(bccfast::k_bcc_energy<3, 2>); break;
      default: go(bccfast::k_bcc_energy<4, 2>); break;
    }
  } else {
    switch (K) {
      case 1: go(bccfast::k_bcc_energy<1, 3>); break;
      case 2: go(bccfast::k_bcc_energy<2, 3>); break;
      case 3: go(bccfast::k_bcc_energy<3, 3>); break;
      default: go(bccfast::k_bcc_energy<4, 3>); break;
    }
  }
  check_cuda(cudaGetLastError(), "tiled energy launch");
  return true;
}

}  // namespace smcx
