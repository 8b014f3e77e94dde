// Sweep kernels.
//
//  * k_tile_sweep  -- tiled generalized checkerboard: one CTA per tile of one
//    tile colour stages the tile plus its interaction halo in shared memory,
//    runs all L^3 m intra-colour phases of the tile with a CTA barrier
//    between phases, and writes the tile plus the one-cell partner ring back.
//    Launched once per tile colour (8 launches per sweep).
//  * k_linkcell_sweep -- the paper's link-cell schedule (Method
//    "Implementation of SMC-GPU": one thread per link cell i_C, one launch per
//    intra colour i_A), reading neighbours straight from global memory.
//
// Both compute, per trial, the Philox words of the site, the partner along a
// uniformly drawn shell-1 direction, the exact integer energy change from the
// two sites' environments (Method "The EPI and qSRO model", paragraph after
// Eq. Total_EPI) and the Metropolis decision u < thr(dE) (Supplementary,
// acceptance equation).
#include <algorithm>

#include "smcx_device.cuh"

namespace smcx {

// Energy change of swapping the species a at s with b at its partner s':
//   dE = sum_k sum_c W_k[c] (n_k(s)[c] - n_k(s')[c]) + X,
//   W_k[c] = V_k[b][c] - V_k[a][c],  X = 2 V_1[a][b] - V_1[a][a] - V_1[b][b],
// where n_k(i)[c] counts shell-k neighbours of i with species c (the partner
// included); X removes the s-s' bond, which a swap leaves unchanged.  The
// tile kernel keeps n_k(s) - n_k(s') in byte-packed counters (NW words of
// four species per shell, each byte biased by 0x80 so that the difference
// never borrows across bytes: at most z_k <= 24 either way), so a trial reads
// each neighbour once and the table K*M times.

template <int KIND, int K, int NW>
__global__ void __launch_bounds__(512) k_tile_sweep(const SweepParams P) {
  constexpr int m = cell_sites(KIND);
  constexpr int NV = vec_count(KIND, K);
  constexpr int Z1 = shell_size(KIND, 0);
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_stat[3];

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
  [[maybe_unused]] const int nbox = P.BX * P.BY * P.BZ * m;  // box bytes (bounds checks of the debug build)

  // tile of this CTA: tile colour bits give the parity on each axis
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

  // stage tile + halo (periodic wrap; the halo never exceeds one lattice edge)
  const int h = P.h;
  stage_generic<m>(P, box, t0, ts, h);
  __syncthreads();

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
      const int dir = P.proposal == 1
                          ? phase_direction(P.seed_lo, P.seed_hi, P.sweep, P.replica,
                                            (unsigned)((ti[2] * P.nt[1] + ti[1]) * P.nt[0] + ti[0]), ic, Z1)
                      : P.proposal == 2
                          ? block_direction(P.seed_lo, P.seed_hi, P.sweep, P.replica, P.tc, (unsigned)blockIdx.x >> 1,
                                            ic, Z1)
                          : (int)__umulhi(rd, (uint32_t)Z1);
      const int sp = s + s_poff[b * Z1 + dir];
      const int bp = s_psub[b * Z1 + dir];
      const int sa = ld_chk(box, s, nbox, kDbgTileBox), sb = ld_chk(box, sp, nbox, kDbgTileBox);
      if (sa == sb) {
        same++;
        continue;
      }
      const int32_t* W = s_w + (sa * M + sb) * KM;
      int dE = s_w[MM * KM + sa * M + sb];
      uint32_t hc[K][NW];
#pragma unroll
      for (int k = 0; k < K; k++)
#pragma unroll
        for (int w = 0; w < NW; w++) hc[k][w] = 0x80808080u;
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const uint32_t c = (uint32_t)ld_chk(box, s + s_off[b * NV + j], nbox, kDbgTileBox);
            const uint32_t one = 1u << (8 * (c & 3));
            if (NW == 1 || c < 4) hc[k][0] += one;
            else hc[k][NW - 1] += one;
          }
        }
      }
      {
        int j = 0;
#pragma unroll
        for (int k = 0; k < K; k++) {
#pragma unroll
          for (int q = 0; q < shell_size(KIND, k); q++, j++) {
            const uint32_t c = (uint32_t)ld_chk(box, sp + s_off[bp * NV + j], nbox, kDbgTileBox);
            const uint32_t one = 1u << (8 * (c & 3));
            if (NW == 1 || c < 4) hc[k][0] -= one;
            else hc[k][NW - 1] -= one;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; k++)
#pragma unroll
        for (int c = 0; c < 4 * NW; c++)
          if (c < M) dE += ((int)((hc[k][c >> 2] >> (8 * (c & 3))) & 0xFFu) - 0x80) * W[k * M + c];
      if (metropolis_accept(dE, ru, s_A, P.nA, s_B)) {
        st_chk(box, s, nbox, kDbgTileBox, (int8_t)sb);
        st_chk(box, sp, nbox, kDbgTileBox, (int8_t)sa);
        acc++;
        dsum += dE;
      }
    }
    __syncthreads();
  }

  // write back the tile and the partner ring
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

template <int KIND, int K>
__global__ void __launch_bounds__(256) k_linkcell_sweep(const SweepParams P) {
  constexpr int m = cell_sites(KIND);
  constexpr int Z1 = shell_size(KIND, 0);
  const int L = P.L;
  const int nlx = P.n[0] / L, nly = P.n[1] / L, nlz = P.n[2] / L;
  const long long nlc = (long long)nlx * nly * nlz;
  const long long lc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long trials = 0, acc = 0, same = 0;
  long long dsum = 0;
  if (lc < nlc) {
    const int b = P.ic % m, lcc = P.ic / m;
    const int cx = lcc % L, cy = (lcc / L) % L, cz = lcc / (L * L);
    const int lx = (int)(lc % nlx);
    const long long r = lc / nlx;
    const int ly = (int)(r % nly), lz = (int)(r / nly);
    const int x = lx * L + cx, y = ly * L + cy, z = lz * L + cz;
    const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
    const unsigned long long gid = (((unsigned long long)z * ny + y) * nx + x) * m + b;
    const uint4 rw = attempt_block(gid, P.sweep, P.replica, P.seed_lo, P.seed_hi);
    const uint32_t rd = (gid & 1) ? rw.z : rw.x;
    const uint32_t ru = (gid & 1) ? rw.w : rw.y;
    const int dir = P.proposal == 1   ? phase_direction(P.seed_lo, P.seed_hi, P.sweep, P.replica, 0u, P.ic, Z1)
                    : P.proposal == 2 ? block_direction(P.seed_lo, P.seed_hi, P.sweep, P.replica, 0, 0u, P.ic, Z1)
                                      : (int)__umulhi(rd, (uint32_t)Z1);
    const signed char* pd = P.gp[b][dir];
    const int px = wrap_add(x, pd[0], nx), py = wrap_add(y, pd[1], ny), pz = wrap_add(z, pd[2], nz);
    const int pb = pd[3];
    const unsigned long long pgid = (((unsigned long long)pz * ny + py) * nx + px) * m + pb;
    const int sa = load_site(P.sites, gid, P.storage), sb = load_site(P.sites, pgid, P.storage);
    trials = 1;
    if (sa == sb) {
      same = 1;
    } else {
      const int M = P.M, KM = K * P.M, MM = P.M * P.M;
      const int32_t* W = P.wtab + (sa * M + sb) * KM;
      int dE = __ldg(P.wtab + MM * KM + sa * M + sb);
      int j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
#pragma unroll
        for (int q = 0; q < shell_size(KIND, k); q++, j++) {
          const signed char* d = P.gd[b][j];
          const unsigned long long t =
              (((unsigned long long)wrap_add(z, d[2], nz) * ny + wrap_add(y, d[1], ny)) * nx +
               wrap_add(x, d[0], nx)) * m + d[3];
          dE += __ldg(W + k * M + load_site(P.sites, t, P.storage));
        }
      }
      j = 0;
#pragma unroll
      for (int k = 0; k < K; k++) {
#pragma unroll
        for (int q = 0; q < shell_size(KIND, k); q++, j++) {
          const signed char* d = P.gd[pb][j];
          const unsigned long long t =
              (((unsigned long long)wrap_add(pz, d[2], nz) * ny + wrap_add(py, d[1], ny)) * nx +
               wrap_add(px, d[0], nx)) * m + d[3];
          dE -= __ldg(W + k * M + load_site(P.sites, t, P.storage));
        }
      }
      if (metropolis_accept(dE, ru, P.thr, P.nA, P.thr + kNA)) {
        acc = 1;
        dsum = dE;
        if (P.storage == SMCX_INT8) {
          P.sites[gid] = (uint8_t)sb;
          P.sites[pgid] = (uint8_t)sa;
        } else {
          // no other trial of this phase touches these two bytes
          uint8_t* p0 = P.sites + (gid >> 1);
          *p0 = (gid & 1) ? (uint8_t)((*p0 & 0x0F) | (sb << 4)) : (uint8_t)((*p0 & 0xF0) | sb);
          uint8_t* p1 = P.sites + (pgid >> 1);
          *p1 = (pgid & 1) ? (uint8_t)((*p1 & 0x0F) | (sa << 4)) : (uint8_t)((*p1 & 0xF0) | sa);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    trials += __shfl_down_sync(0xffffffffu, trials, o);
    acc += __shfl_down_sync(0xffffffffu, acc, o);
    same += __shfl_down_sync(0xffffffffu, same, o);
    dsum += __shfl_down_sync(0xffffffffu, dsum, o);
  }
  if ((threadIdx.x & 31) == 0 && trials) {
    atomicAdd(&P.stats[0], trials);
    atomicAdd(&P.stats[1], acc);
    atomicAdd(&P.stats[2], same);
    atomicAdd(&P.stats[3], (unsigned long long)dsum);
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

static void fill_offsets(const smcx_lattice* hd, SweepParams& P, int BX, int BY) {
  const Shells& S = hd->shells;
  const int m = hd->m;
  for (int b = 0; b < m; b++) {
    int B[3];
    basis_of(hd->kind, b, B);
    for (int j = 0; j < S.nv; j++) {
      int d[3], r[3];
      for (int a = 0; a < 3; a++) {
        int p = B[a] + S.v[j][a];
        d[a] = (p >= 0) ? p / 2 : -((-p + 1) / 2);  // floor(p / 2)
        r[a] = p - 2 * d[a];
      }
      int bb = basis_index(hd->kind, r[0], r[1], r[2]);
      P.off[b][j] = ((d[2] * BY + d[1]) * BX + d[0]) * m + (bb - b);
      P.gd[b][j][0] = (signed char)d[0];
      P.gd[b][j][1] = (signed char)d[1];
      P.gd[b][j][2] = (signed char)d[2];
      P.gd[b][j][3] = (signed char)bb;
      if (j < S.z[0]) {
        P.poff[b][j] = P.off[b][j];
        P.psub[b][j] = bb;
        for (int c = 0; c < 4; c++) P.gp[b][j][c] = P.gd[b][j][c];
      }
    }
  }
}

template <int KIND, int K, int NW>
static void launch_sweeps_nw(smcx_lattice* hd, SweepParams& P, int64_t n_sweeps, int n_colours) {
  const smcx_sched& sc = hd->sched;
  cudaStream_t st = hd->stream;
  if (sc.nt[0] == 1 && sc.nt[1] == 1 && sc.nt[2] == 1) {
    if (n_colours != 8) fail(SMCX_E_UNSUPPORTED, "partial sweeps need a tiled schedule");
    const long long nlc = (long long)(P.n[0] / sc.L) * (P.n[1] / sc.L) * (P.n[2] / sc.L);
    const int grid = (int)((nlc + 255) / 256);
    const int nic = sc.L * sc.L * sc.L * hd->m;
    for (int64_t s = 0; s < n_sweeps; s++) {
      P.sweep = hd->sweep_cum + (uint64_t)s;
      for (int ic = 0; ic < nic; ic++) {
        P.ic = ic;
        k_linkcell_sweep<KIND, K><<<grid, 256, 0, st>>>(P);
      }
    }
    check_cuda(cudaGetLastError(), "link-cell sweep launch");
    return;
  }
  constexpr int m = cell_sites(KIND);
  constexpr int NV = vec_count(KIND, K);
  constexpr int Z1 = shell_size(KIND, 0);
  const int nW = P.M * P.M * K * P.M + P.M * P.M;
  const size_t smem = (size_t)(nW + P.nA + kNB + m * NV + 2 * m * Z1) * 4 +
                      (size_t)P.BX * P.BY * P.BZ * m;
  if (smem > 227 * 1024) fail(SMCX_E_UNSUPPORTED, "tile too large for shared memory");
  check_cuda(cudaFuncSetAttribute(k_tile_sweep<KIND, K, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem),
             "tile sweep smem attribute");
  // a phase has up to ceil(tile / L)^3 trials: one thread each (whole warps,
  // at most 512), so that a phase is one round of the CTA
  int slots = 1;
  for (int a = 0; a < 3; a++) slots *= ((P.n[a] + P.nt[a] - 1) / P.nt[a] + P.L - 1) / P.L;
  const int threads = std::min(512, std::max(32, (slots + 31) / 32 * 32));
  for (int64_t s = 0; s < n_sweeps; s++) {
    P.sweep = hd->sweep_cum + (uint64_t)s;
    for (int tc = 0; tc < n_colours; tc++) {
      P.tc = tc;
      const int grid = P.ntc[0] * P.ntc[1] * P.ntc[2];
      k_tile_sweep<KIND, K, NW><<<grid, threads, smem, st>>>(P);
    }
  }
  check_cuda(cudaGetLastError(), "tile sweep launch");
}

template <int KIND, int K>
static void launch_sweeps(smcx_lattice* hd, SweepParams& P, int64_t n_sweeps, int n_colours) {
  if (hd->M <= 4) launch_sweeps_nw<KIND, K, 1>(hd, P, n_sweeps, n_colours);
  else launch_sweeps_nw<KIND, K, 2>(hd, P, n_sweeps, n_colours);
}

void sweep_device(smcx_lattice* hd, int nA, uint64_t seed, int64_t n_sweeps, int n_colours) {
  if (!hd->Wq.empty()) {
    sweep_qsro_device(hd, nA, seed, n_sweeps, n_colours);
    return;
  }
  if (hd->kernel_choice != 1 && fcc_fast_usable(hd)) {
    sweep_fcc_fast(hd, nA, seed, n_sweeps, n_colours);
    return;
  }
  if (hd->kernel_choice != 1 && bcc_fast_usable(hd)) {
    sweep_bcc_fast(hd, nA, seed, n_sweeps, n_colours);
    return;
  }
  SweepParams P;
  memset(&P, 0, sizeof(P));
  const smcx_sched& sc = hd->sched;
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
  P.proposal = hd->proposal;
  P.seed_lo = (uint32_t)seed;
  P.seed_hi = (uint32_t)(seed >> 32);
  fill_offsets(hd, P, P.BX, P.BY);
  const int K = hd->shells.K;
  if (hd->kind == kBCC) {
    switch (K) {
      case 1: launch_sweeps<kBCC, 1>(hd, P, n_sweeps, n_colours); break;
      case 2: launch_sweeps<kBCC, 2>(hd, P, n_sweeps, n_colours); break;
      case 3: launch_sweeps<kBCC, 3>(hd, P, n_sweeps, n_colours); break;
      case 4: launch_sweeps<kBCC, 4>(hd, P, n_sweeps, n_colours); break;
      default: fail(SMCX_E_UNSUPPORTED, "shell count");
    }
  } else {
    switch (K) {
      case 1: launch_sweeps<kFCC, 1>(hd, P, n_sweeps, n_colours); break;
      case 2: launch_sweeps<kFCC, 2>(hd, P, n_sweeps, n_colours); break;
      case 3: launch_sweeps<kFCC, 3>(hd, P, n_sweeps, n_colours); break;
      default: fail(SMCX_E_UNSUPPORTED, "shell count");
    }
  }
}

}  // namespace smcx
